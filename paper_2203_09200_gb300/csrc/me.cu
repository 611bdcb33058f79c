// me.cu -- dense pixel-wise template-matching motion estimation (Sec. 2.2).
//
// For every pixel p of frame t and every past frame t-k the vector v in [-R, R]^2 (p + v inside
// the frame) minimising the template cost
//     C(p, v) = sum over o in [-h, h]^2 of b_t(p+o) * | f_sub_t(p+o) - rec_{t-k}(clamp(p+v+o)) |
// with b_t = 0 outside the frame and past-frame coordinates clamped to the border.  Equal costs
// are resolved by the tie order |v|_1, then v_y, then v_x (the paper gives none).
//
// GB300 design: integer-only, no tensor cores.  Three exact kernels live here: me9_kernel (T = 9,
// warp strips with byte SIMD and packed 16-bit sums; the tile itself is in me9_tile.cuh), the
// general sliding-window box-sum kernel (any T, this paragraph), and rme9_kernel, the RME reverse
// field for T = 9 (end of the file).  Batched engines choose the ME kernel for T = 9 by measurement (both give the same
// vectors).
//
// Box-sum kernel: one CTA owns a TH x TW tile of outputs for one past frame; the current tile
// (plus the template halo) and the past-frame window (plus the search margin) are staged once in
// shared memory.  Candidates are visited in tie order and, for each, the cost of every output in
// the tile comes from a separable sliding-window box sum over
// the masked absolute-difference plane D_v(x) = b_t(x) |f_sub_t(x) - rec(clamp(x+v))|:
//   1. D_v over the (TH+2h) x (TW+2h) region,
//   2. vertical running sums over T rows (column sums),
//   3. horizontal running sums over T columns -> C(p, v),
// so a cost costs O(1) operations instead of T^2.  The running minimum is an exact integer key
// (cost << 9 | position of v in tie order), so the argmin and its tie rule are bit-exact.
#include <type_traits>

#include "me9_tile.cuh"
#include "rfsr_internal.h"

namespace rfsr {

namespace {

using namespace me9k;

constexpr int TH = 32;           // output tile rows
constexpr int TW = 64;           // output tile columns
constexpr int NT = 256;          // threads per CTA
constexpr int RUN = 8;           // rows per vertical running-sum task
constexpr int SEG = 8;           // columns per horizontal running-sum task
constexpr int CWMAX = TW + 2 * kMaxHalf;
constexpr int CHMAX = TH + 2 * kMaxHalf;
constexpr int RWMAX = CWMAX + 2 * kMaxRadius;
constexpr int RHMAX = CHMAX + 2 * kMaxRadius;

static_assert(TH * (TW / SEG) == NT, "one horizontal task per thread");

struct Smem {
    uint8_t cs[CHMAX * CWMAX];    // current sample plane (unmeasured = 0)
    uint8_t cm[CHMAX * CWMAX];    // current byte mask (0x00 / 0xff)
    uint8_t rf[RHMAX * RWMAX];    // past frame, clamped coordinates
    uint8_t d[CHMAX * CWMAX];     // D_v
    uint16_t col[TH * CWMAX];     // vertical sums
    short2 vord[NVMAX];           // candidates in tie order
};

__device__ __forceinline__ void me_tile(Smem &sm, const FrameTask &t, int tbx, int tby, int k)
{
    const int x0 = tbx * TW, y0 = tby * TH;
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

__global__ void __launch_bounds__(NT) me_kernel(FrameTask t)
{
    __shared__ Smem sm;
    me_tile(sm, t, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Tile of the single-stream launch: 4 warp strips of 8 rows (32-row tiles, four CTAs per SM)
// measured 0.672 ms per 1080p frame, against 0.716 / 0.728 / 0.712 / 0.696 ms for 8 / 6 / 5 / 3
// strips of 8 rows, and 0.83 - 1.0 ms for strips of 12 or 16 rows (168 registers, 12 warps per
// SM).
constexpr int kMeWarps = 4;
constexpr int kMeRows = 8;                   // output rows per warp strip
constexpr int kMeMinBlocks = 16 / kMeWarps;  // resident CTAs the register budget is set for

__global__ void __launch_bounds__(s_nt<kMeWarps>(), kMeMinBlocks) me9_kernel(FrameTask t)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    me9_tile<kMeWarps, kMeRows>(*reinterpret_cast<Smem9<kMeWarps, kMeRows> *>(smem_raw), t,
                                blockIdx.x, blockIdx.y, blockIdx.z);
}

// batched forms on the tile queue: tiles of a task flattened as (k, by, bx), bx fastest
__global__ void __launch_bounds__(NT) me_batched_kernel(BatchDesc *bd)
{
    __shared__ Smem sm;
    __shared__ FrameTask task;
    __shared__ int claim[2];
    claim_tiles(bd, kPhMe, task, claim, [&](const FrameTask &t, int l) {
        const int tx = (t.W + TW - 1) / TW, ty = (t.H + TH - 1) / TH;
        me_tile(sm, t, l % tx, (l / tx) % ty, l / (tx * ty));
    });
}

template <int WARPS>
__global__ void __launch_bounds__(s_nt<WARPS>(), 16 / WARPS) me9_batched_kernel(BatchDesc *bd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem9<WARPS> &sm = *reinterpret_cast<Smem9<WARPS> *>(smem_raw);
    __shared__ FrameTask task;
    __shared__ int claim[2];
    claim_tiles(bd, kPhMe, task, claim, [&](const FrameTask &t, int l) {
        const int tx = (t.W + S_OUTW - 1) / S_OUTW, ty = (t.H + s_outh<WARPS>() - 1) / s_outh<WARPS>();
        me9_tile<WARPS>(sm, t, l % tx, (l / tx) % ty, l / (tx * ty));
    });
}

// ---------------------------------------------------------------------------------------------
// RME reverse field (Sec. 2.2) for T = 9: at every past-frame pixel q the reverse vector
//     w*(q) = argmin over w in [-R, R]^2 with q + w inside the frame of C(q + w, -w),
// costs compared as exact mean costs SAD/n (cross multiplication), the tie order applied to w.
// C(q + w, -w) = sum over o of b_t(q+w+o) |f_sub_t(q+w+o) - rec(clamp(q+o))|: the past-frame patch
// around q stays fixed and the current frame slides, so the warp-strip layout above applies with
// the roles swapped.  A lane keeps 16 rows of the past frame (clamped) in registers; the current
// masked samples and byte masks are staged in shared memory and read shifted by w.  The template
// count n(q + w) differs between candidates: a count plane over the sources of the tile is built
// once from the staged mask, with n = 0 where the source lies outside the frame (so those
// candidates never win).  The running best of an output is one word:
//     SAD (15 bits) | tie position of w (9 bits) << 15 | n (7 bits) << 24.
// ---------------------------------------------------------------------------------------------
constexpr int R9_OUTH = S_ROWS * 8;                        // tile rows (8 warps)
constexpr int R9_NT = 256;
constexpr int R9_SROWS = R9_OUTH + 8 + 2 * kMaxRadius;     // staged current-frame rows
constexpr int R9_NROWS = R9_OUTH + 2 * kMaxRadius;         // count-plane rows (source rows)
constexpr int R9_RB = 4 * S_RWORDS;                        // bytes per staged row

struct SmemR9 {
    union {
        uint32_t c[R9_SROWS * S_RWORDS];                   // current masked samples
        uint8_t hs[R9_SROWS * R9_RB];                      // horizontal mask sums (set-up only)
    };
    uint32_t m[R9_SROWS * S_RWORDS];                       // current byte masks
    uint32_t n[R9_NROWS * S_RWORDS];                       // template counts at the sources
    short2 vord[NVMAX];
};

// staged row r, byte b of word w = pixel (ry0 + r, rx0 + 4w + b) of src, 0 outside the frame
__device__ __forceinline__ void stage_current(uint32_t *dst, const uint8_t *__restrict__ src, int H,
                                              int W, int ry0, int rx0, int nrows)
{
    for (int i = threadIdx.x; i < nrows * S_RWORDS; i += R9_NT) {
        const int r = i / S_RWORDS, w = i - r * S_RWORDS;
        const int y = ry0 + r, gx = rx0 + 4 * w;
        uint32_t v = 0;
        if (y >= 0 && y < H) {
            const uint8_t *row = src + (size_t)y * W;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int x = gx + b;
                if (x >= 0 && x < W) v |= (uint32_t)row[x] << (8 * b);
            }
        }
        dst[i] = v;
    }
}

__device__ __forceinline__ void rme9_tile(SmemR9 &sm, const FrameTask &t, int tbx, int tby, int k)
{
    const int x0 = tbx * S_OUTW, y0 = tby * R9_OUTH;
    const int H = t.H, W = t.W, R = t.R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*t.status) return;
    const uint8_t *__restrict__ ref = t.ref_rec[k];
    const int rx0 = x0 - 4 - R, ry0 = y0 - 4 - R;            // staged origin
    const int nrows = R9_OUTH + 8 + 2 * R, ncnt = R9_OUTH + 2 * R;

    // 1. byte masks of the current frame around the tile, and the tie order
    stage_current(sm.m, t.cur_msk, H, W, ry0, rx0, nrows);
    build_tie_order(sm.vord, R);
    __syncthreads();
    // 2. horizontal 9-sums of the mask bits at staged columns 4 .. R9_RB - 5
    const uint8_t *mb = reinterpret_cast<const uint8_t *>(sm.m);
    for (int i = tid; i < nrows * (R9_RB - 8); i += R9_NT) {
        const int r = i / (R9_RB - 8), col = 4 + i - r * (R9_RB - 8);
        int s = 0;
#pragma unroll
        for (int dx = -4; dx <= 4; ++dx) s += mb[r * R9_RB + col + dx] & 1;
        sm.hs[r * R9_RB + col] = (uint8_t)s;
    }
    __syncthreads();
    // 3. template counts n at the sources (row y0 - R + rr, column rx0 + col); 0 outside the frame
    uint8_t *nb = reinterpret_cast<uint8_t *>(sm.n);
    for (int i = tid; i < R9_NROWS * R9_RB; i += R9_NT) {
        const int rr = i / R9_RB, col = i - rr * R9_RB;
        const int sy = y0 - R + rr, sx = rx0 + col;
        int v = 0;
        if (rr < ncnt && col >= 4 && col < R9_RB - 4 && sy >= 0 && sy < H && sx >= 0 && sx < W) {
#pragma unroll
            for (int j = 0; j < 9; ++j) v += sm.hs[(rr + j) * R9_RB + col];
        }
        nb[i] = (uint8_t)v;
    }
    __syncthreads();
    // 4. masked samples of the current frame (over the horizontal sums)
    stage_current(sm.c, t.cur_smp, H, W, ry0, rx0, nrows);
    // 5. this lane's 16 past-frame rows of 4 columns, clamped coordinates
    const int cx = x0 - 4 + 4 * lane;
    const int cy0 = y0 + S_ROWS * warp - 4;
    uint32_t fr[S_DROWS];
#pragma unroll
    for (int i = 0; i < S_DROWS; ++i) {
        const uint8_t *row = ref + (size_t)min(max(cy0 + i, 0), H - 1) * W;
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) v |= (uint32_t)row[min(max(cx + b, 0), W - 1)] << (8 * b);
        fr[i] = v;
    }
    __syncthreads();

    uint32_t best[S_ROWS][4];
#pragma unroll
    for (int j = 0; j < S_ROWS; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) best[j][c] = 0x7fffu | (1u << 24);   // "infinite", n = 1
    const int nv = (2 * R + 1) * (2 * R + 1);
    const uint32_t one = (uint32_t)(W > 0), m1 = 0u - one;  // 1 and -1 (W > 0 always)
    for (int o = 0; o < nv; ++o) {
        const short2 w = sm.vord[o];
        const int wy = w.x, wx = w.y;
        const int sh = (wx + R) & 3, q = (wx + R) >> 2;
        const uint32_t sel = 0x3210u + 0x1111u * (uint32_t)sh;
        const int base = (S_ROWS * warp + wy + R) * S_RWORDS + lane + q;
        const uint32_t *crow = sm.c + base, *mrow = sm.m + base, *nrow = sm.n + base;
        const uint32_t o15 = (uint32_t)o << 15;
        uint32_t lo = 0, hi = 0;
        uint32_t dlo[S_DROWS], dhi[S_DROWS];
#pragma unroll
        for (int i = 0; i < S_DROWS; ++i) {
            const uint32_t c4 = __byte_perm(crow[i * S_RWORDS], crow[i * S_RWORDS + 1], sel);
            const uint32_t m4 = __byte_perm(mrow[i * S_RWORDS], mrow[i * S_RWORDS + 1], sel);
            const uint32_t d4 = __vabsdiffu4(fr[i], c4) & m4;
            dlo[i] = __byte_perm(d4, 0u, 0x4240);
            dhi[i] = __byte_perm(d4, 0u, 0x4341);
            lo = imad(dlo[i], one, lo);
            hi = imad(dhi[i], one, hi);
            if (i >= 9) {
                lo = imad(dlo[i - 9], m1, lo);
                hi = imad(dhi[i - 9], m1, hi);
            }
            if (i >= 8) {
                const int j = i - 8;                       // output row of this window
                const uint32_t Q = imad(hi, one, lo);
                const uint32_t Ql = __shfl_up_sync(0xffffffffu, Q, 1);
                const uint32_t lol = __shfl_up_sync(0xffffffffu, lo, 1);
                const uint32_t Qr = __shfl_down_sync(0xffffffffu, Q, 1);
                const uint32_t lor = __shfl_down_sync(0xffffffffu, lo, 1);
                const uint32_t A = __byte_perm(Ql, Q, 0x5432);
                const uint32_t B = __byte_perm(Q, Qr, 0x5432);
                const uint32_t h02 = imad(lor, one, imad(imad(B, one, Q), one, imad(A, one, Ql)));
                const uint32_t h13 = imad(imad(lol, m1, Qr), one, imad(lor, m1, h02));
                const uint32_t n4 = __byte_perm(nrow[j * S_RWORDS], nrow[j * S_RWORDS + 1], sel);
                const uint32_t sad[4] = {h02 & 0xffffu, h13 & 0xffffu, h02 >> 16, h13 >> 16};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t n = (n4 >> (8 * c)) & 0xffu;
                    const uint32_t b = best[j][c];
                    const bool take = sad[c] * (b >> 24) < (b & 0x7fffu) * n;
                    best[j][c] = take ? (sad[c] | o15 | (n << 24)) : b;
                }
            }
        }
    }
    if (lane == 0 || lane == 31) return;
    char2 *rmv = reinterpret_cast<char2 *>(t.rmv[k]);
    const int oy = y0 + S_ROWS * warp;
#pragma unroll
    for (int j = 0; j < S_ROWS; ++j) {
        const int y = oy + j;
        if (y >= H) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int x = cx + c;
            if (x < W) {
                const short2 w = sm.vord[(best[j][c] >> 15) & 0x1ffu];
                rmv[(size_t)y * W + x] = make_char2((signed char)w.x, (signed char)w.y);
            }
        }
    }
}

__global__ void __launch_bounds__(R9_NT, 2) rme9_kernel(FrameTask t)
{
    __shared__ SmemR9 sm;
    rme9_tile(sm, t, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(R9_NT, 2) rme9_batched_kernel(BatchDesc *bd)
{
    __shared__ SmemR9 sm;
    __shared__ FrameTask task;
    __shared__ int claim[2];
    claim_tiles(bd, kPhRme, task, claim, [&](const FrameTask &t, int l) {
        const int tx = (t.W + S_OUTW - 1) / S_OUTW, ty = (t.H + R9_OUTH - 1) / R9_OUTH;
        rme9_tile(sm, t, l % tx, (l / tx) % ty, l / (tx * ty));
    });
}

// ---------------------------------------------------------------------------------------------
// Predictive-centre search for references k >= 2 (an opt-in variant that the paper does not
// describe; it changes the method's results).  Motion to frame t-k is predicted as k v_1(p),
// v_1 the exact vector to frame t-1, and only the window of radius Rp around that prediction is
// searched, within [-R, R]^2 so that every later stage keeps its layout:
//     c = (clamp(k v_1y, max(-R, -y), min(R, H-1-y)), clamp(k v_1x, max(-R, -x), min(R, W-1-x)))
//     v_k(p) = argmin over v in (c + [-Rp, Rp]^2) n [-R, R]^2 with p + v inside the frame of
//              C(p, v), the same cost and tie order as the full search (Sec. 2.2).
// The clamp keeps p + c inside the frame, so the centre is always a candidate, and Rp >= 2R
// covers the whole window: the result is then the full search's.
// GB300 design: one CTA per 32x32 output tile and reference, the current frame and the past
// frame (with its +-9 margin) staged in four byte-shifted copies.  Each pixel has its own window,
// so the candidate sharing of the full search does not carry over directly.  Most pixels of a
// tile share one predicted centre, however (coherent motion), and for the most frequent centre
// c* of a tile, if at least P_DENSE_MIN pixels have it, the window c* + [-Rp, Rp]^2 is searched
// densely: each warp takes some of its candidates and computes the candidate's cost at every
// tile pixel by separable 9 x 9 box sums of the masked absolute-difference plane (the forward
// ME's packed vertical sums and shuffle horizontal sums), keeping per pixel the smallest key
// SAD << 9 | tie position; the warps' keys meet in shared memory (atomicMin).  The other pixels
// are searched one by one: a thread keeps the pixel's template (masked samples and byte masks,
// 9 rows of 3 words) in registers and scores its window with `vabsdiff4.add` per word.
// ---------------------------------------------------------------------------------------------
constexpr int P_TS = 32;                           // output tile side
constexpr int P_NT = 256;
constexpr int P_NW = P_NT / 32;
constexpr int P_RROWS = P_TS + 8 + 2 * kMaxRadius + 2;   // staged past-frame rows (60; the dense
                                                   // pass's third row band reads one row past)
constexpr int P_RWORDS = 17;                       // words per staged past-frame row (from x0 - 16)
constexpr int P_RCPY = P_RROWS * P_RWORDS + 12;    // copy stride = 8 (mod 32) words: the four
                                                   // copies of one word lie in distinct banks
constexpr int P_CROWS = P_TS + 8 + 2;              // staged current rows (42, likewise)
constexpr int P_CWORDS = 11;                       // words per staged current row (from x0 - 4)
constexpr int P_DENSE_MIN = 128;                   // pixels of one centre that pay for a dense pass
constexpr int P_HS = 2 * kMaxRadius + 1;
static_assert(P_RCPY % 32 == 8, "past-frame copy stride");
static_assert((P_TS - 1) + 12 + kMaxRadius + 11 < 4 * (P_RWORDS - 1), "shifted past-frame words cover the reads");

// The tie order (|v|_1, v_y, v_x) over [-9, 9]^2, built at compile time: position of every v and
// the vector at every position.  Restricted to [-R, R]^2 it keeps its relative order, so it
// ranks the candidates of every R.
struct TieTables {
    uint16_t rank[P_HS * P_HS];                    // bin (v_y + 9) * 19 + v_x + 9 -> position
    uint16_t bin[P_HS * P_HS];                     // position -> bin
};
constexpr TieTables make_tie_tables()
{
    TieTables t{};
    int n = 0;
    for (int L = 0; L <= 2 * kMaxRadius; ++L)
        for (int vy = -kMaxRadius; vy <= kMaxRadius; ++vy) {
            const int ax = L - (vy < 0 ? -vy : vy);
            if (ax < 0 || ax > kMaxRadius) continue;
            for (int s = -1; s <= 1; s += 2) {
                if (ax == 0 && s > 0) break;
                const int b = (vy + kMaxRadius) * P_HS + s * ax + kMaxRadius;
                t.rank[b] = (uint16_t)n;
                t.bin[n++] = (uint16_t)b;
            }
        }
    return t;
}
__constant__ TieTables c_tie = make_tie_tables();

struct SmemP {
    uint32_t rf[4 * P_RCPY];                       // past frame, clamped coordinates
    uint2 cur[4][P_CROWS * P_CWORDS];              // (masked samples, byte mask) words
    TieTables tie;
    uint16_t cen[P_TS * P_TS];                     // predicted centre of each tile pixel (bin)
    uint16_t plist[P_TS * P_TS];                   // pixels searched one by one
    int hist[P_HS * P_HS];                         // tile pixels per centre
    uint32_t dkey[P_TS * P_TS];                    // dense pass: best key per tile pixel
    int cstar;                                     // centre searched densely (bin), -1: none
    int np;
};

__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b, uint32_t acc)
{
    uint32_t d;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(acc));
    return d;
}

// predicted centre of pixel (y, x) for reference distance kk from its t-1 vector p1
__device__ __forceinline__ int pred_centre(char2 p1, int kk, int y, int x, int H, int W, int R)
{
    const int cy = min(max(kk * (int)p1.x, max(-R, -y)), min(R, H - 1 - y));
    const int cx = min(max(kk * (int)p1.y, max(-R, -x)), min(R, W - 1 - x));
    return (cy + kMaxRadius) * P_HS + cx + kMaxRadius;
}

__global__ void __launch_bounds__(P_NT) me_pred_kernel(FrameTask t)
{
    __shared__ __align__(16) SmemP sm;
    const int k = blockIdx.z + 1;                  // reference t-(k+1); its field is t.mv[k]
    const int x0 = blockIdx.x * P_TS, y0 = blockIdx.y * P_TS;
    const int H = t.H, W = t.W, R = t.R, Rp = t.me_pred, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (*t.status) return;
    const uint8_t *ref = t.ref_rec[k];
    const char2 *mv1 = reinterpret_cast<const char2 *>(t.mv[0]);

    // past frame: rows y0 - 4 - 9 .., words from column x0 - 16, clamped coordinates
    const bool al = (W & 3) == 0 && ((uintptr_t)ref & 3) == 0;
    for (int i = tid; i < P_RROWS * P_RWORDS; i += P_NT) {
        const int r = i / P_RWORDS, w = i - r * P_RWORDS;
        const uint8_t *row = ref + (size_t)min(max(y0 - 4 - kMaxRadius + r, 0), H - 1) * W;
        const int gx = x0 - 16 + 4 * w;
        uint32_t v = 0;
        if (al && gx >= 0 && gx + 4 <= W) {
            v = *reinterpret_cast<const uint32_t *>(row + gx);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) v |= (uint32_t)row[min(max(gx + b, 0), W - 1)] << (8 * b);
        }
        sm.rf[i] = v;
    }
    // current frame: rows y0 - 4 .., words from column x0 - 4 (0 outside the frame)
    const bool alc = (W & 3) == 0 && (((uintptr_t)t.cur_smp | (uintptr_t)t.cur_msk) & 3) == 0;
    for (int i = tid; i < P_CROWS * P_CWORDS; i += P_NT) {
        const int r = i / P_CWORDS, w = i - r * P_CWORDS;
        const int gy = y0 - 4 + r, gx = x0 - 4 + 4 * w;
        uint32_t a = 0, m = 0;
        if (gy >= 0 && gy < H) {
            const size_t ro = (size_t)gy * W;
            if (alc && gx >= 0 && gx + 4 <= W) {       // gx is a multiple of 4
                a = *reinterpret_cast<const uint32_t *>(t.cur_smp + ro + gx);
                m = *reinterpret_cast<const uint32_t *>(t.cur_msk + ro + gx);
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int x = gx + b;
                    if (x >= 0 && x < W) {
                        a |= (uint32_t)t.cur_smp[ro + x] << (8 * b);
                        m |= (uint32_t)t.cur_msk[ro + x] << (8 * b);
                    }
                }
            }
        }
        sm.cur[0][i] = make_uint2(a, m);
    }
    for (int i = tid; i < P_HS * P_HS; i += P_NT) {
        sm.hist[i] = 0;
        sm.tie.rank[i] = c_tie.rank[i];
        sm.tie.bin[i] = c_tie.bin[i];
    }
    if (tid == 0) sm.np = 0;
    __syncthreads();
    for (int i = tid; i < 3 * P_RROWS * (P_RWORDS - 1); i += P_NT) {
        const int j = 1 + i / (P_RROWS * (P_RWORDS - 1));
        const int rem = i - (j - 1) * P_RROWS * (P_RWORDS - 1);
        const int r = rem / (P_RWORDS - 1), w = rem - r * (P_RWORDS - 1);
        sm.rf[j * P_RCPY + r * P_RWORDS + w] =
            __funnelshift_r(sm.rf[r * P_RWORDS + w], sm.rf[r * P_RWORDS + w + 1], 8 * j);
    }
    for (int i = tid; i < 3 * P_CROWS * (P_CWORDS - 1); i += P_NT) {
        const int j = 1 + i / (P_CROWS * (P_CWORDS - 1));
        const int rem = i - (j - 1) * P_CROWS * (P_CWORDS - 1);
        const int r = rem / (P_CWORDS - 1), w = rem - r * (P_CWORDS - 1);
        const uint2 a = sm.cur[0][r * P_CWORDS + w], b = sm.cur[0][r * P_CWORDS + w + 1];
        sm.cur[j][r * P_CWORDS + w] = make_uint2(__funnelshift_r(a.x, b.x, 8 * j),
                                                 __funnelshift_r(a.y, b.y, 8 * j));
    }
    // predicted centres and their histogram (lanes with the same centre add up first)
    for (int pi = tid; pi < P_TS * P_TS; pi += P_NT) {
        const int py = pi / P_TS, px = pi - py * P_TS, y = y0 + py, x = x0 + px;
        uint32_t c = 0xffffu;
        if (y < H && x < W) c = (uint32_t)pred_centre(mv1[(size_t)y * W + x], k + 1, y, x, H, W, R);
        const unsigned same = __match_any_sync(0xffffffffu, c);
        if (c != 0xffffu && lane == __ffs(same) - 1) atomicAdd(&sm.hist[c], __popc(same));
        sm.cen[pi] = (uint16_t)c;
        sm.dkey[pi] = 0xffffffffu;
    }
    __syncthreads();
    if (warp == 0) {                               // the most frequent centre
        uint32_t key = 0;                          // count << 10 | 1023 - bin
        for (int i = lane; i < P_HS * P_HS; i += 32)
            key = max(key, ((uint32_t)sm.hist[i] << 10) | (1023u - i));
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0) sm.cstar = (int)(key >> 10) >= P_DENSE_MIN ? 1023 - (int)(key & 1023u) : -1;
    }
    __syncthreads();
    const int cstar = sm.cstar;

    // dense pass over the window of c*: lanes 0..29 are three bands of 11 rows x 10 words (the
    // 8 words of the tile and a halo word on each side), one candidate at a time per warp
    if (cstar >= 0) {
        const int csy = cstar / P_HS - kMaxRadius, csx = cstar % P_HS - kMaxRadius;
        const int ch = min(lane / 10, 2), wi = lane < 30 ? lane - 10 * ch : 9, r0 = 11 * ch;
        const bool out = lane < 30 && wi >= 1 && wi <= 8;
        const bool inner = y0 - R >= 0 && x0 - R >= 0 && y0 + P_TS + R <= H && x0 + P_TS + R <= W;
        uint32_t best[11][4];
#pragma unroll
        for (int j = 0; j < 11; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) best[j][c] = 0xffffffffu;
        const int side = 2 * Rp + 1;
        for (int i = warp; i < side * side; i += P_NW) {
            const int vy = csy + i / side - Rp, vx = csx + i % side - Rp;
            if (vy < -R || vy > R || vx < -R || vx > R) continue;      // uniform over the warp
            const uint32_t rk = c_tie.rank[(vy + kMaxRadius) * P_HS + vx + kMaxRadius];
            const uint32_t *rr = sm.rf + ((vx + 12) & 3) * P_RCPY + (r0 + vy + kMaxRadius) * P_RWORDS +
                                 wi + ((vx + 12) >> 2);
            const uint2 *cc = sm.cur[0] + r0 * P_CWORDS + wi;
            uint32_t dlo[19], dhi[19], lo = 0, hi = 0;
#pragma unroll
            for (int q = 0; q < 19; ++q) {
                const uint2 c = cc[q * P_CWORDS];
                const uint32_t d4 = __vabsdiffu4(c.x, rr[q * P_RWORDS]) & c.y;
                dlo[q] = __byte_perm(d4, 0u, 0x4240);
                dhi[q] = __byte_perm(d4, 0u, 0x4341);
                lo += dlo[q];
                hi += dhi[q];
                if (q >= 9) {
                    lo -= dlo[q - 9];
                    hi -= dhi[q - 9];
                }
                if (q >= 8) {
                    const int j = q - 8;                   // output row r0 + j
                    const uint32_t Q = lo + hi;
                    const uint32_t Ql = __shfl_up_sync(0xffffffffu, Q, 1);
                    const uint32_t lol = __shfl_up_sync(0xffffffffu, lo, 1);
                    const uint32_t Qr = __shfl_down_sync(0xffffffffu, Q, 1);
                    const uint32_t lor = __shfl_down_sync(0xffffffffu, lo, 1);
                    const uint32_t A = __byte_perm(Ql, Q, 0x5432), B = __byte_perm(Q, Qr, 0x5432);
                    const uint32_t h02 = Ql + A + Q + B + lor;
                    const uint32_t h13 = h02 + Qr - lol - lor;
                    const uint32_t h[4] = {h02 & 0xffffu, h13 & 0xffffu, h02 >> 16, h13 >> 16};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int y = y0 + r0 + j, x = x0 + 4 * (wi - 1) + c;
                        const bool ok = inner || ((unsigned)(y + vy) < (unsigned)H &&
                                                  (unsigned)(x + vx) < (unsigned)W);
                        if (ok) best[j][c] = min(best[j][c], (h[c] << 9) | rk);
                    }
                }
            }
        }
        if (out) {
#pragma unroll
            for (int j = 0; j < 11; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int py = r0 + j, px = 4 * (wi - 1) + c;
                    if (py < P_TS && sm.cen[py * P_TS + px] == (uint16_t)cstar)
                        atomicMin(&sm.dkey[py * P_TS + px], best[j][c]);
                }
        }
        __syncthreads();
    }

    // densely searched pixels are done; the others are listed and searched one per thread
    char2 *mvk = reinterpret_cast<char2 *>(t.mv[k]);
    auto store = [&](int pi, uint32_t key) {
        const int b = sm.tie.bin[key & 511u];
        mvk[(size_t)(y0 + pi / P_TS) * W + x0 + pi % P_TS] =
            make_char2((signed char)(b / P_HS - kMaxRadius), (signed char)(b % P_HS - kMaxRadius));
    };
    for (int pi = tid; pi < P_TS * P_TS; pi += P_NT) {
        const int cb = sm.cen[pi];
        if (cb == 0xffff) continue;                // outside the frame
        if (cb == cstar) store(pi, sm.dkey[pi]);
        else sm.plist[atomicAdd(&sm.np, 1)] = (uint16_t)pi;
    }
    __syncthreads();
    const int np = sm.np;
    for (int e = tid; e < np; e += P_NT) {
        const int pi = sm.plist[e], py = pi / P_TS, px = pi - py * P_TS, y = y0 + py, x = x0 + px;
        const int cb = sm.cen[pi];
        uint32_t cs[9][3], cm[9][3];               // template: masked samples and byte masks
#pragma unroll
        for (int r = 0; r < 9; ++r)
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                const uint2 c = sm.cur[px & 3][(py + r) * P_CWORDS + (px >> 2) + w];
                const uint32_t keep = w == 2 ? 0xffu : 0xffffffffu;   // template columns 0..8
                cs[r][w] = c.x & keep;
                cm[r][w] = c.y & keep;
            }
        const int cy = cb / P_HS - kMaxRadius, cx = cb % P_HS - kMaxRadius;
        uint32_t best = 0xffffffffu;               // SAD << 9 | position in the tie order
        for (int vy = max(cy - Rp, -R); vy <= min(cy + Rp, R); ++vy) {
            if ((unsigned)(y + vy) >= (unsigned)H) continue;
            for (int vx = max(cx - Rp, -R); vx <= min(cx + Rp, R); ++vx) {
                if ((unsigned)(x + vx) >= (unsigned)W) continue;
                const int rc = px + 12 + vx;      // staged column of the template's first byte
                const uint32_t *rr = sm.rf + (rc & 3) * P_RCPY + (py + vy + kMaxRadius) * P_RWORDS + (rc >> 2);
                uint32_t acc = 0;
#pragma unroll
                for (int r = 0; r < 9; ++r)
#pragma unroll
                    for (int w = 0; w < 3; ++w) acc = sad4(cs[r][w], rr[r * P_RWORDS + w] & cm[r][w], acc);
                best = min(best, (acc << 9) | sm.tie.rank[(vy + kMaxRadius) * P_HS + vx + kMaxRadius]);
            }
        }
        store(pi, best);
    }
}

}  // namespace

cudaError_t init_me(int dev)
{
    static int ready[64] = {};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (ready[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(me9_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem9<kMeWarps, kMeRows>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(me9_batched_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Smem9<8>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(me9_batched_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Smem9<4>));
    if (e == cudaSuccess) ready[dev] = 1;
    return e;
}

int tiles_me(const FrameTask &t, int me_warps, int me_box)
{
    if (t.K <= 0) return 0;
    const int outh = S_ROWS * me_warps;
    if (t.T == 9 && !me_box) return ((t.W + S_OUTW - 1) / S_OUTW) * ((t.H + outh - 1) / outh) * t.K;
    return ((t.W + TW - 1) / TW) * ((t.H + TH - 1) / TH) * t.K;
}

cudaError_t launch_me(const FrameTask &t, cudaStream_t st)
{
    if (t.K <= 0) return cudaSuccess;
    if (t.T == 9) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = init_me(dev);
        if (e != cudaSuccess) return e;
        constexpr int outh = s_outh<kMeWarps, kMeRows>();
        // predictive-centre variant: the full search for t-1 only, then the windows around k v_1
        const bool pred = t.me_pred > 0 && t.K > 1;
        dim3 grid((t.W + S_OUTW - 1) / S_OUTW, (t.H + outh - 1) / outh, pred ? 1 : t.K);
        me9_kernel<<<grid, s_nt<kMeWarps>(), sizeof(Smem9<kMeWarps, kMeRows>), st>>>(t);
        if (pred) {
            count_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            dim3 pgrid((t.W + P_TS - 1) / P_TS, (t.H + P_TS - 1) / P_TS, t.K - 1);
            me_pred_kernel<<<pgrid, P_NT, 0, st>>>(t);
        }
    } else {
        dim3 grid((t.W + TW - 1) / TW, (t.H + TH - 1) / TH, t.K);
        me_kernel<<<grid, NT, 0, st>>>(t);
    }
    count_launch();
    return cudaGetLastError();
}

int tiles_rme9(const FrameTask &t)
{
    if (t.K <= 0) return 0;
    return ((t.W + S_OUTW - 1) / S_OUTW) * ((t.H + R9_OUTH - 1) / R9_OUTH) * t.K;
}

cudaError_t launch_rme9(const FrameTask &t, cudaStream_t st)
{
    if (t.K <= 0) return cudaSuccess;
    dim3 grid((t.W + S_OUTW - 1) / S_OUTW, (t.H + R9_OUTH - 1) / R9_OUTH, t.K);
    rme9_kernel<<<grid, R9_NT, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rme9_batched(BatchDesc *bd, cudaStream_t st)
{
    static std::atomic<int> grids[64];
    const int grid = persistent_grid_cached(rme9_batched_kernel, R9_NT, 0, grids);
    rme9_batched_kernel<<<grid, R9_NT, 0, st>>>(bd);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_me_batched(BatchDesc *bd, int T, int me_warps, int me_box, cudaStream_t st)
{
    if (T == 9 && me_box) T = 0;                 // the box-sum kernel below handles any T
    if (T == 9) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = init_me(dev);
        if (e != cudaSuccess) return e;
    }
    if (T == 9 && me_warps == 4) {
        static std::atomic<int> grids[64];
        const int grid = persistent_grid_cached(me9_batched_kernel<4>, s_nt<4>(), sizeof(Smem9<4>), grids);
        me9_batched_kernel<4><<<grid, s_nt<4>(), sizeof(Smem9<4>), st>>>(bd);
    } else if (T == 9) {
        static std::atomic<int> grids[64];
        const int grid = persistent_grid_cached(me9_batched_kernel<8>, s_nt<8>(), sizeof(Smem9<8>), grids);
        me9_batched_kernel<8><<<grid, s_nt<8>(), sizeof(Smem9<8>), st>>>(bd);
    } else {
        static std::atomic<int> grids[64];
        const int grid = persistent_grid_cached(me_batched_kernel, NT, 0, grids);
        me_batched_kernel<<<grid, NT, 0, st>>>(bd);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
