// me.cu -- dense pixel-wise template-matching motion estimation (Sec. 2.2).
//
// For every pixel p of frame t and every past frame t-k the vector v in [-R, R]^2 (p + v inside
// the frame) minimising the template cost
//     C(p, v) = sum over o in [-h, h]^2 of b_t(p+o) * | f_sub_t(p+o) - rec_{t-k}(clamp(p+v+o)) |
// with b_t = 0 outside the frame and past-frame coordinates clamped to the border.  Equal costs
// are resolved by the tie order |v|_1, then v_y, then v_x (the paper gives none).
//
// GB300 design: integer-only, no tensor cores.  One CTA owns a TH x TW tile of outputs for one
// past frame; the current tile (plus the template halo) and the past-frame window (plus the
// search margin) are staged once in shared memory.  Candidates are visited in tie order and, for
// each, the cost of every output in the tile comes from a separable sliding-window box sum over
// the masked absolute-difference plane D_v(x) = b_t(x) |f_sub_t(x) - rec(clamp(x+v))|:
//   1. D_v over the (TH+2h) x (TW+2h) region,
//   2. vertical running sums over T rows (column sums),
//   3. horizontal running sums over T columns -> C(p, v),
// so a cost costs O(1) operations instead of T^2.  The running minimum is an exact integer key
// (cost << 9 | position of v in tie order), so the argmin and its tie rule are bit-exact.
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int TH = 32;           // output tile rows
constexpr int TW = 64;           // output tile columns
constexpr int NT = 256;          // threads per CTA
constexpr int RUN = 8;           // rows per vertical running-sum task
constexpr int SEG = 8;           // columns per horizontal running-sum task
constexpr int CWMAX = TW + 2 * kMaxHalf;
constexpr int CHMAX = TH + 2 * kMaxHalf;
constexpr int RWMAX = CWMAX + 2 * kMaxRadius;
constexpr int RHMAX = CHMAX + 2 * kMaxRadius;
constexpr int NVMAX = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);

static_assert(TH * (TW / SEG) == NT, "one horizontal task per thread");

struct Smem {
    uint8_t cs[CHMAX * CWMAX];    // current sample plane (unmeasured = 0)
    uint8_t cm[CHMAX * CWMAX];    // current byte mask (0x00 / 0xff)
    uint8_t rf[RHMAX * RWMAX];    // past frame, clamped coordinates
    uint8_t d[CHMAX * CWMAX];     // D_v
    uint16_t col[TH * CWMAX];     // vertical sums
    short2 vord[NVMAX];           // candidates in tie order
};

// Candidates of [-R, R]^2 sorted by (|v|_1, v_y, v_x): enumerate |v|_1 = L, then v_y ascending,
// then v_x ascending (-|v_x| before +|v_x|).
__device__ void build_tie_order(short2 *vord, int R)
{
    if (threadIdx.x != 0) return;
    int n = 0;
    for (int L = 0; L <= 2 * R; ++L)
        for (int vy = -R; vy <= R; ++vy) {
            const int ax = L - (vy < 0 ? -vy : vy);
            if (ax < 0 || ax > R) continue;
            vord[n++] = make_short2((short)vy, (short)-ax);
            if (ax != 0) vord[n++] = make_short2((short)vy, (short)ax);
        }
}

__global__ void __launch_bounds__(NT) me_kernel(FrameTask t)
{
    __shared__ Smem sm;
    const int k = blockIdx.z;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int H = t.H, W = t.W, T = t.T, h = t.T / 2, R = t.R;
    const int CW = TW + 2 * h, CH = TH + 2 * h;
    const int RW = CW + 2 * R, RH = CH + 2 * R;
    const uint8_t *__restrict__ ref = t.ref_rec[k];
    const int tid = threadIdx.x;

    if (*t.status) return;   // bad mask in this frame: leave everything untouched

    for (int i = tid; i < CH * CW; i += NT) {
        const int ry = i / CW, rx = i - ry * CW;
        const int gy = y0 - h + ry, gx = x0 - h + rx;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sm.cs[i] = in ? t.cur_smp[(size_t)gy * W + gx] : 0;
        sm.cm[i] = in ? t.cur_msk[(size_t)gy * W + gx] : 0;
    }
    for (int i = tid; i < RH * RW; i += NT) {
        const int ry = i / RW, rx = i - ry * RW;
        const int gy = min(max(y0 - h - R + ry, 0), H - 1);
        const int gx = min(max(x0 - h - R + rx, 0), W - 1);
        sm.rf[i] = ref[(size_t)gy * W + gx];
    }
    build_tie_order(sm.vord, R);
    __syncthreads();

    const int nv = (2 * R + 1) * (2 * R + 1);
    const int by = tid / (TW / SEG), bxs = (tid % (TW / SEG)) * SEG;   // horizontal task
    const int gy = y0 + by;
    uint32_t best[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i) best[i] = 0xffffffffu;

    for (int o = 0; o < nv; ++o) {
        const short2 v = sm.vord[o];
        // 1. D_v over the region
        for (int i = tid; i < CH * CW; i += NT) {
            const int ry = i / CW, rx = i - ry * CW;
            const int a = sm.cs[i];
            const int b = sm.rf[(ry + R + v.x) * RW + rx + R + v.y];
            sm.d[i] = (uint8_t)(sm.cm[i] & (a > b ? a - b : b - a));
        }
        __syncthreads();
        // 2. vertical running sums: column c, output rows [ys, ys + RUN)
        for (int task = tid; task < CW * (TH / RUN); task += NT) {
            const int c = task % CW, ys = (task / CW) * RUN;
            int acc = 0;
            for (int dy = 0; dy < T; ++dy) acc += sm.d[(ys + dy) * CW + c];
            sm.col[ys * CWMAX + c] = (uint16_t)acc;
            for (int y = ys + 1; y < ys + RUN; ++y) {
                acc += sm.d[(y + T - 1) * CW + c] - sm.d[(y - 1) * CW + c];
                sm.col[y * CWMAX + c] = (uint16_t)acc;
            }
        }
        __syncthreads();
        // 3. horizontal running sums and the running argmin
        {
            const uint16_t *row = sm.col + by * CWMAX;
            int acc = 0;
            for (int dx = 0; dx < T; ++dx) acc += row[bxs + dx];
            const bool row_ok = (unsigned)(gy + v.x) < (unsigned)H;
#pragma unroll
            for (int i = 0; i < SEG; ++i) {
                if (i > 0) acc += row[bxs + i + T - 1] - row[bxs + i - 1];
                const int gx = x0 + bxs + i;
                const bool ok = row_ok && (unsigned)(gx + v.y) < (unsigned)W;
                const uint32_t key = ((uint32_t)acc << 9) | (uint32_t)o;
                if (ok) best[i] = min(best[i], key);
            }
        }
        __syncthreads();
    }
    if (gy < H) {
        char2 *mv = reinterpret_cast<char2 *>(t.mv[k]);
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            const int gx = x0 + bxs + i;
            if (gx < W) {
                const short2 v = sm.vord[best[i] & 511u];
                mv[(size_t)gy * W + gx] = make_char2((signed char)v.x, (signed char)v.y);
            }
        }
    }
}

}  // namespace

cudaError_t launch_me(const FrameTask &t, cudaStream_t st)
{
    if (t.K <= 0) return cudaSuccess;
    dim3 grid((t.W + TW - 1) / TW, (t.H + TH - 1) / TH, t.K);
    me_kernel<<<grid, NT, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
