// cc.cu -- consistency checks and projection (Sec. 2.2, Sec. 3.1).
//
// For each pixel p of frame t and each past frame t-k (k = 1..K):
//   v~  = component-wise 3x3 median of the ME field (Eq. (1), border replicated) when the mode
//         includes NNC, else the raw vector;  q = p + v~
//   MEASURED        if p is measured in frame t
//   NOT_PROJECTABLE if q is outside the frame or not measured in frame t-k (only measurements
//                   are projected, Sec. 2.2)
//   NNC_REJECT      if the NNC is on and some in-frame 4-neighbour u has |v~(p)-v~(u)|_1 > 1
//                   (Sec. 3.1.2)
//   CHECK_REJECT    if the reverse check fails:
//                     FRMC: some reverse vector -v~+d, d in {-7,-3,-1,0,1,3,7}^2, has a strictly
//                           lower cost than d = 0 (Sec. 3.1.1, Fig. 2c)
//                     RMC:  the same with d in [-Rc, Rc]^2 (Fig. 2b)
//                     RME:  the reverse motion vector found at q is not -v~ (Sec. 2.2)
//                   the reverse cost of d is C(p+d, v~-d): the current-frame template slides
//                   around p while the past-frame patch around q stays fixed; costs are compared
//                   as exact mean absolute differences SAD/n (cross multiplication)
//   ACCEPT          otherwise: psum(p) += f_sub_{t-k}(q), pcnt(p) += 1
// The projected value psum/pcnt is the average over the past frames that project (Sec. 2.2).
// NNC runs first and the reverse check only for NNC survivors (the combination of Sec. 3.1.2).
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int iabs(int v) { return v < 0 ? -v : v; }

// template cost C(src, v) against the past frame: SAD over measured current-frame pixels of the
// T x T window around src, past-frame coordinates clamped.  n = number of measured pixels.
__device__ void cost_at(const FrameTask &t, const uint8_t *__restrict__ ref, int sy, int sx,
                        int vy, int vx, int &sad, int &n)
{
    const int h = t.T / 2, H = t.H, W = t.W;
    int s = 0, c = 0;
    for (int oy = -h; oy <= h; ++oy) {
        const int y = sy + oy;
        if ((unsigned)y >= (unsigned)H) continue;
        const int ry = min(max(y + vy, 0), H - 1);
        const uint8_t *crow = t.cur_smp + (size_t)y * W;
        const uint8_t *mrow = t.cur_msk + (size_t)y * W;
        const uint8_t *rrow = ref + (size_t)ry * W;
        for (int ox = -h; ox <= h; ++ox) {
            const int x = sx + ox;
            if ((unsigned)x >= (unsigned)W || !mrow[x]) continue;
            const int rx = min(max(x + vx, 0), W - 1);
            s += iabs((int)crow[x] - (int)rrow[rx]);
            c += 1;
        }
    }
    sad = s;
    n = c;
}

// a = (sa, na) strictly lower mean cost than b = (sb, nb)
__device__ __forceinline__ bool lower(int sa, int na, int sb, int nb)
{
    return (long long)sa * nb < (long long)sb * na;
}

__device__ __forceinline__ bool tie_before(int ay, int ax, int by, int bx)
{
    const int la = iabs(ay) + iabs(ax), lb = iabs(by) + iabs(bx);
    if (la != lb) return la < lb;
    if (ay != by) return ay < by;
    return ax < bx;
}

// RMC / FRMC: accept iff no tested reverse vector has a strictly lower cost than d = 0
__device__ bool reverse_check(const FrameTask &t, const uint8_t *__restrict__ ref, int py, int px,
                              int vy, int vx, bool fast)
{
    const int fset[7] = {-7, -3, -1, 0, 1, 3, 7};
    int s0, n0;
    cost_at(t, ref, py, px, vy, vx, s0, n0);
    const int nset = fast ? 7 : 2 * t.Rc + 1;
    for (int i = 0; i < nset; ++i) {
        const int dy = fast ? fset[i] : i - t.Rc;
        const int sy = py + dy;
        if ((unsigned)sy >= (unsigned)t.H) continue;
        for (int j = 0; j < nset; ++j) {
            const int dx = fast ? fset[j] : j - t.Rc;
            if (dy == 0 && dx == 0) continue;
            const int sx = px + dx;
            if ((unsigned)sx >= (unsigned)t.W) continue;
            int s, n;
            cost_at(t, ref, sy, sx, vy - dy, vx - dx, s, n);
            if (lower(s, n, s0, n0)) return false;
        }
    }
    return true;
}

// median of nine values: sort each group of three, then the median of (largest minimum,
// median of medians, smallest maximum) -- exact for any input, ties included.
__device__ __forceinline__ void cswap(int &a, int &b)
{
    const int lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

__device__ __forceinline__ int med3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

__device__ int median9(int p0, int p1, int p2, int p3, int p4, int p5, int p6, int p7, int p8)
{
    cswap(p0, p1); cswap(p1, p2); cswap(p0, p1);
    cswap(p3, p4); cswap(p4, p5); cswap(p3, p4);
    cswap(p6, p7); cswap(p7, p8); cswap(p6, p7);
    const int lo = max(max(p0, p3), p6);
    const int hi = min(min(p2, p5), p8);
    return med3(lo, med3(p1, p4, p7), hi);
}

__device__ __forceinline__ char2 load_mv(const char2 *mv, int H, int W, int y, int x)
{
    y = min(max(y, 0), H - 1);
    x = min(max(x, 0), W - 1);
    return mv[(size_t)y * W + x];
}

__device__ void median_vec(const char2 *mv, int H, int W, int y, int x, int &my, int &mx)
{
    char2 a[9];
    int c = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) a[c++] = load_mv(mv, H, W, y + dy, x + dx);
    my = median9(a[0].x, a[1].x, a[2].x, a[3].x, a[4].x, a[5].x, a[6].x, a[7].x, a[8].x);
    mx = median9(a[0].y, a[1].y, a[2].y, a[3].y, a[4].y, a[5].y, a[6].y, a[7].y, a[8].y);
}

__global__ void __launch_bounds__(NT) cc_project_kernel(FrameTask t)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
    if (x >= t.W || y >= t.H || *t.status) return;
    const int H = t.H, W = t.W;
    const size_t i = (size_t)y * W + x;
    const bool use_nnc = t.cc_mode == 4 || t.cc_mode == 5;
    const bool measured = t.cur_msk[i] != 0;
    int sum = 0, cnt = 0;
    for (int k = 0; k < t.K; ++k) {
        const char2 *mv = reinterpret_cast<const char2 *>(t.mv[k]);
        int fy, fx;
        bool pass = true;
        if (use_nnc) {
            median_vec(mv, H, W, y, x, fy, fx);
            const int nb[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int yy = y + nb[j][0], xx = x + nb[j][1];
                if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)W) continue;
                int ny, nx;
                median_vec(mv, H, W, yy, xx, ny, nx);
                if (iabs(fy - ny) + iabs(fx - nx) > 1) pass = false;
            }
        } else {
            const char2 v = mv[i];
            fy = v.x;
            fx = v.y;
        }
        reinterpret_cast<char2 *>(t.fmv[k])[i] = make_char2((signed char)fy, (signed char)fx);
        const int qy = y + fy, qx = x + fx;
        uint8_t d;
        if (measured) {
            d = 0;                                               // MEASURED
        } else if ((unsigned)qy >= (unsigned)H || (unsigned)qx >= (unsigned)W ||
                   !t.ref_msk[k][(size_t)qy * W + qx]) {
            d = 1;                                               // NOT_PROJECTABLE
        } else if (use_nnc && !pass) {
            d = 2;                                               // NNC_REJECT
        } else {
            bool ok = true;
            if (t.cc_mode == 3 || t.cc_mode == 5) ok = reverse_check(t, t.ref_rec[k], y, x, fy, fx, true);
            else if (t.cc_mode == 2) ok = reverse_check(t, t.ref_rec[k], y, x, fy, fx, false);
            else if (t.cc_mode == 1) {
                const char2 w = reinterpret_cast<const char2 *>(t.rmv[k])[(size_t)qy * W + qx];
                ok = (w.x == -fy) && (w.y == -fx);
            }
            d = ok ? 4 : 3;                                      // ACCEPT / CHECK_REJECT
        }
        t.dec[k][i] = d;
        if (d == 4) {
            sum += t.ref_smp[k][(size_t)qy * W + qx];
            cnt += 1;
        }
    }
    t.psum[i] = (uint16_t)sum;
    t.pcnt[i] = (uint8_t)cnt;
}

// RME (Sec. 2.2): reverse motion vector at every past-frame pixel q: argmin over w in [-R, R]^2
// with q + w inside of C(q + w, -w), exact mean-cost order, tie order on w.
__global__ void __launch_bounds__(NT) rme_field_kernel(FrameTask t)
{
    const int qx = blockIdx.x * 32 + (threadIdx.x & 31);
    const int qy = blockIdx.y * (NT / 32) + (threadIdx.x >> 5);
    const int k = blockIdx.z;
    if (qx >= t.W || qy >= t.H || *t.status) return;
    const int R = t.R;
    int bs = 0, bn = 0, by = 0, bx = 0;
    bool have = false;
    for (int wy = -R; wy <= R; ++wy) {
        const int sy = qy + wy;
        if ((unsigned)sy >= (unsigned)t.H) continue;
        for (int wx = -R; wx <= R; ++wx) {
            const int sx = qx + wx;
            if ((unsigned)sx >= (unsigned)t.W) continue;
            int s, n;
            cost_at(t, t.ref_rec[k], sy, sx, -wy, -wx, s, n);
            const long long l = (long long)s * bn, r = (long long)bs * n;
            if (!have || l < r || (l == r && tie_before(wy, wx, by, bx))) {
                bs = s; bn = n; by = wy; bx = wx; have = true;
            }
        }
    }
    reinterpret_cast<char2 *>(t.rmv[k])[(size_t)qy * t.W + qx] = make_char2((signed char)by, (signed char)bx);
}

}  // namespace

cudaError_t launch_cc_project(const FrameTask &t, cudaStream_t st)
{
    dim3 grid((t.W + 31) / 32, (t.H + NT / 32 - 1) / (NT / 32));
    cc_project_kernel<<<grid, NT, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rme_field(const FrameTask &t, cudaStream_t st)
{
    if (t.K <= 0) return cudaSuccess;
    dim3 grid((t.W + 31) / 32, (t.H + NT / 32 - 1) / (NT / 32), t.K);
    rme_field_kernel<<<grid, NT, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
