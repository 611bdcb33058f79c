// fsr.cu -- block-wise frequency selective reconstruction (Sec. 2.1) with projected pixels as
// additional known pixels and the D-FSR overwrite rule (Sec. 3.2); concealed weighting is zero
// (Sec. 4) so every 4x4 block depends only on measured / projected pixels of its 32x32 support
// and all blocks of a frame run in parallel.  The 8-bit reconstruction that becomes the next
// frame's reference is written in the same kernel.
//
// Model (the standard FSR matching-pursuit loop; the paper defers its details to the literature):
//   known pixel: measured (value s/255, weight rho^d) or projected (value psum/(255 pcnt),
//   weight mu rho^d), d = distance to the support centre; all other pixels weight 0.
//   W = DFT(weights), R = DFT(weights * values); per iteration the conjugate pair u maximising
//   wf(u) |R(u)|^2 is selected (ties: lower canonical linear index), dc = gamma R(u) / W(0), and
//       g += dc phi_u + conj(dc) phi_-u,      R(k) -= dc W(k-u) + conj(dc) W(k+u)
//   (self-conjugate u: g += Re(dc) phi_u, R(k) -= Re(dc) W(k-u)).  Output: g at the 16 block
//   pixels, measured pixels overwritten by their samples (and, for R-FSR, projected pixels by
//   their projected value).
//
// GB300 design: one warp per block, FP32.
//   * DFTs by FFT: each lane transforms one support row (32 real values as a 16-point complex
//     radix-2 FFT plus the real-input split), then one column of the half spectrum (32-point
//     complex radix-2 FFT, in place in shared memory); twiddles come from a host-computed table
//     in constant memory at compile-time indices.
//   * R is Hermitian (the signal is real), so 17 bins per lane suffice: rows 0..16 at columns
//     0..16 and rows 1..15 at columns 16..32, in registers with their frequency weights.  The
//     full weight spectrum W (read at shifts k -+ u) lives in shared memory as rows of 49 columns
//     (0..31 and 0..16 again), so both shifted reads are immediate offsets from one pointer and
//     the 32 lanes' row-shifted reads fall in distinct banks.
//   * Selection: per lane a max tree over integer keys (the float bits of e with the slot in the
//     low 5 bits), the warp maximum from __reduce_max_sync and the lowest canonical index among
//     the lanes that reach it from __reduce_min_sync.  The winning bin's slot is the same in
//     every lane, so the owner lane reads R there through one uniform switch and a shuffle pair
//     sends it out.
//     The rank-2 residual update works on (Re, Im) as packed FP32 pairs
//     (R -= dr (a + c) + di (c.y - a.y, a.x - c.x)): one pair add, two scalar subtractions and two
//     pair FMAs per bin.
//   * The per-warp shared memory is one 12.5 KB union (support, row spectra, W).
#include <cmath>
#include <type_traits>

#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int N = kFsrN;
constexpr int NH = kFsrHalf;
constexpr int WPB1 = 4;                    // warps (blocks) per CTA of the single-stream launch
constexpr int WC = N + NH;                 // W row with wrap-around: column c holds W(., c mod 32)
constexpr int WS = WC;                     // row stride of W (float2); 49 -> rows 2 banks apart
constexpr int SS = N + 1;                  // padded row stride of the support (float)

__constant__ float c_cs[N];                // cos(2 pi j / 32)
__constant__ float c_sn[N];                // sin(2 pi j / 32)

union WarpSmem {
    struct {
        float w[N * SS];                   // support weights
        float f[N * SS];                   // weighted values
    } sup;
    struct {
        float2 w[N * NH];                  // row spectra of the weights, then column pass in place
        float2 f[N * NH];                  // row spectra of the weighted values
    } dft;
    float2 W[N * WS + NH];                 // full weight spectrum, columns 0..48 (wrapped),
                                           // then a zero row (the second term of a self-
                                           // conjugate update)
};

// the fields of a FrameTask that the FSR of one block reads
struct FsrArgs {
    const uint8_t *msk, *smp;              // current mask (0x00 / 0xFF) and masked samples
    const uint16_t *psum;                  // projection sums and counts (null: none)
    const uint8_t *pcnt;
    float *fsr_out;                        // optional outputs
    uint8_t *rec, *out_u8;
    const FsrTables *tab;
    const int *status;
    int *status_out;
    const float *conc;                     // concealed weighting: this frame's output so far
    uint16_t *sel;                         // optional trace: selected pair per block and iteration
    int H, W, iters, overwrite;
    float gamma, mu, delta;
};

__device__ __forceinline__ void fsr_args(FsrArgs &a, const FrameTask &t)
{
    a.msk = t.cur_msk;
    a.smp = t.cur_smp;
    a.psum = t.psum;
    a.pcnt = t.pcnt;
    a.fsr_out = t.fsr_out;
    a.rec = t.cur_rec;
    a.out_u8 = t.out_u8;
    a.tab = reinterpret_cast<const FsrTables *>(t.fsr_tables);
    a.status = t.status;
    a.status_out = t.status_out;
    a.H = t.H;
    a.W = t.W;
    a.iters = t.fsr_iters;
    a.overwrite = t.fsr_overwrite_projected;
    a.gamma = t.fsr_gamma;
    a.mu = t.fsr_proj_weight;
    a.conc = t.fsr_out;
    a.delta = t.fsr_concealed;
    a.sel = t.fsr_sel;
}

struct Twiddles {
    float cs[N];
    float sn[N];
};

template <int WPB>                         // WPB blocks (one per warp) per CTA
struct Smem {
    Twiddles tw;
    FsrArgs args[WPB];                     // batched kernel: each warp's current task
    int tile[2];                           // batched kernel: claimed tiles (double-buffered)
    WarpSmem w[WPB];
};

__host__ __device__ constexpr int bitrev(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E), so that every register
// array index below is a constant expression
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// in-place radix-2 decimation-in-time FFT (forward, exp(-2 pi i k n / M)) of M points given in
// bit-reversed order; twiddle W_M^j = cos(2 pi j/M) - i sin(2 pi j/M) = table index j * 32 / M
template <int M, int LEN = 2>
__device__ __forceinline__ void fft_dit(float (&re)[M], float (&im)[M])
{
    if constexpr (LEN <= M) {
        static_for<0, M / 2>([&](auto q) {
            constexpr int Q = decltype(q)::value;
            constexpr int i = (Q / (LEN / 2)) * LEN, j = Q % (LEN / 2);
            constexpr int a = i + j, b = i + j + LEN / 2;
            constexpr int tw = j * (N / LEN);
            float xr, xi;
            if constexpr (tw == 0) {
                xr = re[b];
                xi = im[b];
            } else if constexpr (tw == N / 4) {         // -i
                xr = im[b];
                xi = -re[b];
            } else {
                const float wr = c_cs[tw], wi = -c_sn[tw];
                xr = re[b] * wr - im[b] * wi;
                xi = re[b] * wi + im[b] * wr;
            }
            re[b] = re[a] - xr;
            im[b] = im[a] - xi;
            re[a] += xr;
            im[a] += xi;
        });
        fft_dit<M, 2 * LEN>(re, im);
    }
}

// DFT of one 32-point real row x (natural order) -> X[0..16], via a 16-point complex FFT of
// z[n] = x[2n] + i x[2n+1] and X[l] = E[l] + W_32^l O[l] with E, O the even / odd spectra
__device__ __forceinline__ void real_row_dft(const float (&x)[N], float2 *out)
{
    float zr[16], zi[16];
    static_for<0, 16>([&](auto nn) {
        constexpr int n = decltype(nn)::value;
        zr[bitrev(n, 4)] = x[2 * n];
        zi[bitrev(n, 4)] = x[2 * n + 1];
    });
    fft_dit<16>(zr, zi);
    static_for<0, 17>([&](auto ll) {
        constexpr int l = decltype(ll)::value;
        constexpr int a = l & 15, b = (16 - l) & 15;
        const float ar = zr[a], ai = zi[a], br = zr[b], bi = -zi[b];   // Z[l], conj(Z[16-l])
        const float er = 0.5f * (ar + br), ei = 0.5f * (ai + bi);       // E = (Z + conj Z') / 2
        const float orr = 0.5f * (ai - bi), oi = -0.5f * (ar - br);     // O = (Z - conj Z') / 2i
        float tr, ti;
        if constexpr (l == 0 || l == 16) {                              // W = +1 / -1
            tr = l == 0 ? orr : -orr;
            ti = l == 0 ? oi : -oi;
        } else if constexpr (l == 8) {                                  // W = -i
            tr = oi;
            ti = -orr;
        } else {
            const float wr = c_cs[l], wi = -c_sn[l];
            tr = orr * wr - oi * wi;
            ti = orr * wi + oi * wr;
        }
        out[l] = make_float2(er + tr, ei + ti);
    });
}

// 32-point complex DFT of column c of a [32][17] array, in place
__device__ __forceinline__ void column_dft(float2 *a, int c)
{
    float re[N], im[N];
    static_for<0, N>([&](auto mm) {
        constexpr int m = decltype(mm)::value;
        const float2 v = a[m * NH + c];
        re[bitrev(m, 5)] = v.x;
        im[bitrev(m, 5)] = v.y;
    });
    fft_dit<N>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) a[k * NH + c] = make_float2(re[k], im[k]);
}

// 32-point complex DFTs of columns c and c + 1 of a [32][17] array, in place, by the whole warp:
// lane m holds element m of both; radix-2 decimation in frequency over shuffles leaves X[k] in
// lane bitrev(k).  Every lane runs the same instructions (the butterfly's sum and its twiddled
// difference are both formed and one is kept), with the twiddles from the shared-memory table.
__device__ __forceinline__ void warp_column_dft2(float2 *a, int c, const float *cs, const float *sn,
                                                 int lane)
{
    float2 x = a[lane * NH + c], y = a[lane * NH + c + 1];
#pragma unroll
    for (int h = N / 2; h >= 1; h >>= 1) {
        const float xr = __shfl_xor_sync(0xffffffffu, x.x, h), xi = __shfl_xor_sync(0xffffffffu, x.y, h);
        const float yr = __shfl_xor_sync(0xffffffffu, y.x, h), yi = __shfl_xor_sync(0xffffffffu, y.y, h);
        const bool upper = (lane & h) != 0;               // element b of its butterfly
        const int j = (lane & (h - 1)) * (N / (2 * h));   // W_{2h}^(t - h) = W_32^j
        const float wr = cs[j], wi = -sn[j];
        const float dxr = xr - x.x, dxi = xi - x.y, dyr = yr - y.x, dyi = yi - y.y;
        x = upper ? make_float2(dxr * wr - dxi * wi, dxr * wi + dxi * wr) : make_float2(x.x + xr, x.y + xi);
        y = upper ? make_float2(dyr * wr - dyi * wi, dyr * wi + dyi * wr) : make_float2(y.x + yr, y.y + yi);
    }
    const int k = (int)(__brev((unsigned)lane) >> (32 - 5));
    a[k * NH + c] = x;
    a[k * NH + c + 1] = y;
}

// Support row m (frame row y) at support column `lane` (frame column x) of block (bi, bj): the
// weight rho^d (x mu for projected pixels, x delta for concealed ones) and the weighted value.
__device__ __forceinline__ void support_row(WarpSmem &ws, const FsrArgs &a, int m, int x, int y,
                                            int bi, int bj, int lane)
{
    float wt = 0.f, val = 0.f;
    if ((unsigned)x < (unsigned)a.W && (unsigned)y < (unsigned)a.H) {
        const size_t i = (size_t)y * a.W + x;
        const float wd = __ldg(&a.tab->wsp[m * N + lane]);
        const unsigned mk = __ldg(a.msk + i), sv = __ldg(a.smp + i);
        const unsigned c = a.pcnt != nullptr ? __ldg(a.pcnt + i) : 0u;
        const unsigned ps = a.pcnt != nullptr ? __ldg(a.psum + i) : 0u;
        if (mk) {
            wt = wd;
            val = (float)sv * (1.0f / 255.0f);
        } else if (c) {
            wt = a.mu * wd;
            val = (float)ps / (255.0f * (float)c);
        } else if (a.delta > 0.f && (y / kFsrB < bi || (y / kFsrB == bi && x / kFsrB < bj))) {
            wt = a.delta * wd;                   // reconstructed earlier (raster order)
            val = a.conc[i];
        }
    }
    ws.sup.w[m * SS + lane] = wt;
    ws.sup.f[m * SS + lane] = wt * val;
}

// output of one block pixel: D-FSR overwrite (R-FSR also overwrites projected pixels) and the
// 8-bit reconstruction
__device__ __forceinline__ void store_pixel(const FsrArgs &a, int y, int x, float g)
{
    if (y >= a.H || x >= a.W) return;
    const size_t i = (size_t)y * a.W + x;
    float v = g;
    uint8_t q;
    if (a.msk[i]) {
        v = (float)a.smp[i] * (1.0f / 255.0f);
        q = a.smp[i];
    } else {
        if (a.overwrite && a.pcnt != nullptr && a.pcnt[i])
            v = (float)a.psum[i] / (255.0f * (float)a.pcnt[i]);
        const float r = rintf(255.0f * v);
        q = (uint8_t)fminf(fmaxf(r, 0.0f), 255.0f);
    }
    if (a.fsr_out) a.fsr_out[i] = v;
    if (a.rec) a.rec[i] = q;
    if (a.out_u8) a.out_u8[i] = q;
}

// block b of a frame, computed by one warp with its shared-memory area ws; tw holds the
// twiddles.  Block 0 also publishes the frame's final status word.  TRACE: the instantiation
// that also records the selected pair of every iteration in a.sel (when it is set).
template <bool TRACE>
__device__ __forceinline__ void fsr_block(const Twiddles &tw, WarpSmem &ws, const FsrArgs &a, int b)
{
    const int lane = threadIdx.x & 31;
    const int status = *a.status;
    if (b == 0 && lane == 0 && a.status_out != nullptr) *a.status_out = status;
    if (status) return;

    const int H = a.H, W = a.W;
    const int nbx = (W + kFsrB - 1) / kFsrB, nby = (H + kFsrB - 1) / kFsrB;
    if (b >= nbx * nby) return;
    const int bi = b / nbx, bj = b - bi * nbx;
    const int o = (N - kFsrB) / 2;
    const int ys = kFsrB * bi - o, xs = kFsrB * bj - o;
    const int iters = a.iters;
    const float gamma = a.gamma;
    const FsrTables *tab = a.tab;

    // 1. support: lane = column, coalesced row loads; rows unrolled so that their loads overlap
    {
        const int x = xs + lane;
#pragma unroll 4
        for (int m = 0; m < N; ++m) support_row(ws, a, m, x, ys + m, bi, bj, lane);
    }
    __syncwarp();

    // 2. row DFTs: lane = support row
    {
        float xw[N], xf[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            xw[n] = ws.sup.w[lane * SS + n];
            xf[n] = ws.sup.f[lane * SS + n];
        }
        __syncwarp();                                  // the union is rewritten below
        real_row_dft(xw, &ws.dft.w[lane * NH]);
        real_row_dft(xf, &ws.dft.f[lane * NH]);
    }
    __syncwarp();

    // 3. column DFTs in place: 34 columns (17 of W, then 17 of R): one per lane, and the last two
    //    by the whole warp together, rather than by two lanes while the other 30 wait
    column_dft(lane < NH ? ws.dft.w : ws.dft.f, lane < NH ? lane : lane - NH);
    warp_column_dft2(ws.dft.f, N - NH, tw.cs, tw.sn, lane);
    __syncwarp();

    // 4. 17 bins of the half spectrum per lane in registers.  Lane k <= 16 holds R(k, s), lane
    //    k > 16 holds R(32 - k, 16 + s) = conj(R(k, 16 - s)), s = 0..16.  Slot s then has the
    //    canonical linear index rowbase + s in every lane (the bins (32 - k, 16) and (32 - k, 0)
    //    of slots 0 and 16 in lanes k > 16 repeat bins of lane 32 - k and get weight 0), so a tie
    //    inside a lane always goes to the lowest slot.  W goes to the full padded layout.
    const int k = lane;
    const bool upper = k > N / 2;
    const int kap = upper ? N - k : k;                 // row of the held bins
    const int c0 = upper ? N / 2 : 0;                  // column of slot 0
    const int rowbase = kap * N + c0;                  // canonical linear index of slot 0
    float2 Rr[NH];                                     // (Re, Im) of R(kap, c0 + s)
    {
        float2 Wt[NH];
#pragma unroll
        for (int s = 0; s < NH; ++s) {
            const float2 r = ws.dft.f[k * NH + (upper ? NH - 1 - s : s)];
            Rr[s] = upper ? make_float2(r.x, -r.y) : r;
            Wt[s] = ws.dft.w[k * NH + s];
        }
        __syncwarp();
#pragma unroll
        for (int l = 0; l < NH; ++l) ws.W[k * WS + l] = Wt[l];
    }
    __syncwarp();
    // W(k, l) for l = 17..31 from Hermitian symmetry, W(k, l) = conj(W(-k, -l)); columns 32..48
    // repeat 0..16 so that the shifted reads W(kap -+ u, c0 + s -+ u_l) need no wrap-around
#pragma unroll
    for (int l = NH; l < N; ++l) {
        const float2 a = ws.W[((N - k) & (N - 1)) * WS + (N - l)];
        ws.W[k * WS + l] = make_float2(a.x, -a.y);
    }
#pragma unroll
    for (int l = 0; l < NH; ++l) ws.W[k * WS + N + l] = ws.W[k * WS + l];
    if (lane < NH) ws.W[N * WS + lane] = make_float2(0.f, 0.f);
    __syncwarp();
    const float W0 = ws.W[0].x;

    // frequency weights of the held bins (wf is even in both frequencies), 0 for the repeats
    float wfr[NH];
#pragma unroll
    for (int s = 0; s < NH; ++s) {
        const bool held = !upper || (s != 0 && s != NH - 1);
        wfr[s] = held ? __ldg(&tab->wf[k * NH + (upper ? NH - 1 - s : s)]) : 0.f;
    }

    const int pm = (lane >> 2) & 3, pn = lane & 3;     // block pixel of lanes 0..15
    const int jm = o + pm, jn = o + pn;
    float g = 0.f;
    const float gscale = W0 > 0.f ? gamma / W0 : 0.f;
    // the model term of the previous iteration, added while this iteration's reductions run:
    // g += gf (dr cos - di sin) at phase jp (gf = 1 for a self-conjugate bin, else 2)
    float gdr = 0.f, gdi = 0.f, gf = 0.f;
    int jp = 0;
    int it = 0;
    for (; it < iters && W0 > 0.f; ++it) {
        // Selection key of slot s: the bits of e = wf |R|^2 (e >= 0, so they order like e) with
        // the low 5 bits replaced by 31 - s.  The integer maximum then picks the largest e and,
        // among values equal to 2^-18 relative, the lowest slot; a max tree keeps the scan short.
        uint32_t key[NH];
#pragma unroll
        for (int s = 0; s < NH; ++s) {
            const float e = wfr[s] * fmaf(Rr[s].x, Rr[s].x, Rr[s].y * Rr[s].y);
            key[s] = (__float_as_uint(e) & ~31u) | (uint32_t)(31 - s);
        }
#pragma unroll
        for (int w = 1; w < NH; w *= 2)
#pragma unroll
            for (int s = 0; s + w < NH; s += 2 * w) key[s] = max(key[s], key[s + w]);
        const uint32_t best = key[0];
        const int cand = rowbase + 31 - (int)(best & 31);   // canonical index of the lane's best
        g = fmaf(gf, fmaf(gdr, tw.cs[jp], -gdi * tw.sn[jp]), g);
        const uint32_t m = __reduce_max_sync(0xffffffffu, best);
        gf = 0.f;
        if ((m >> 5) == 0) break;                      // residual exhausted
        // among the lanes whose value reaches the maximum, the lowest canonical index wins
        const int mykey = ((best ^ m) >> 5) == 0 ? cand : 0x7fffffff;
        const int win = __reduce_min_sync(0xffffffffu, mykey);
        if constexpr (TRACE) {
            if (a.sel != nullptr && lane == 0) a.sel[(size_t)b * iters + it] = (uint16_t)win;
        }
        const int uk = win >> 5, ul = win & (N - 1);   // the canonical bin u
        // R(u) from its owner: lane uk, slot ul (ul <= 16) or lane 32 - uk, slot ul - 16; the
        // slot is the same in every lane, so one switch branch reads it
        const int owner = ul <= N / 2 ? uk : N - uk;
        const int slot = ul <= N / 2 ? ul : ul - N / 2;
        float2 rv = Rr[0];
        switch (slot) {
#define RFSR_CASE(c) case c: rv = Rr[c]; break;
            RFSR_CASE(1) RFSR_CASE(2) RFSR_CASE(3) RFSR_CASE(4) RFSR_CASE(5) RFSR_CASE(6)
            RFSR_CASE(7) RFSR_CASE(8) RFSR_CASE(9) RFSR_CASE(10) RFSR_CASE(11) RFSR_CASE(12)
            RFSR_CASE(13) RFSR_CASE(14) RFSR_CASE(15) RFSR_CASE(16)
#undef RFSR_CASE
            default: break;
        }
        const float ure = __shfl_sync(0xffffffffu, rv.x, owner);
        const float uim = __shfl_sync(0xffffffffu, rv.y, owner);
        const bool self = ((uk & (N / 2 - 1)) == 0) && ((ul & (N / 2 - 1)) == 0);
        const float dr = gscale * ure;
        const float di = self ? 0.f : gscale * uim;
        // W(kap - u) and W(kap + u) of the held bins start at columns (c0 -+ u_l) mod 32; a
        // self-conjugate u has no second term, so its second read is the zero row
        const float2 *pa = ws.W + ((kap - uk) & (N - 1)) * WS + ((c0 - ul) & (N - 1));
        const float2 *pc = self ? ws.W + N * WS
                                : ws.W + ((kap + uk) & (N - 1)) * WS + ((c0 + ul) & (N - 1));
        // packed FP32 pairs: R -= dr (a + c) + di (c.y - a.y, a.x - c.x)
        const float2 ndr = make_float2(-dr, -dr), ndi = make_float2(-di, -di);
#pragma unroll
        for (int l = 0; l < NH; ++l) {
            const float2 a = pa[l], c = pc[l];
            const float2 s = __fadd2_rn(a, c);
            const float2 q = make_float2(c.y - a.y, a.x - c.x);
            Rr[l] = __ffma2_rn(ndi, q, __ffma2_rn(ndr, s, Rr[l]));
        }
        // model at the block pixel of this lane, added in the next iteration (or after the loop)
        jp = (uk * jm + ul * jn) & (N - 1);
        gdr = dr;
        gdi = di;
        gf = self ? 1.f : 2.f;
    }
    g = fmaf(gf, fmaf(gdr, tw.cs[jp], -gdi * tw.sn[jp]), g);
    if constexpr (TRACE) {                             // iterations not run: no selection
        if (a.sel != nullptr)
            for (int j = it + lane; j < iters; j += 32) a.sel[(size_t)b * iters + j] = 0xffffu;
    }

    // 5. output: D-FSR overwrite and the 8-bit reconstruction
    if (lane < kFsrB * kFsrB) store_pixel(a, kFsrB * bi + pm, kFsrB * bj + pn, g);
}

// The same block computed by MW warps together (concealed weighting > 0, where blocks run as
// wavefronts and the time is one block's latency, not the throughput of many).  Warp w holds the
// slots s = w + MW j of every lane (slot 16 in warp 0), so a warp scans and updates a quarter of
// the bins.  One barrier per iteration publishes every warp's best key and its lowest canonical
// index among the lanes that reach it (the global winner is the lowest index among the warps
// whose maximum is the global one); a second one publishes R(u) from its owner.  Every bin sees
// the same operations in the same order as in fsr_block, so the results are identical.  (One
// barrier with every warp's candidate R published beside its key measured slower.)
constexpr int MW = 4;                      // warps per block
constexpr int MWS = (NH + MW - 1) / MW;    // slots per lane and warp (the last only in warp 0)

struct MwSmem {
    Twiddles tw;
    WarpSmem ws;
    uint32_t redm[MW];                     // per warp: maximum key
    int redc[MW];                          // per warp: lowest canonical index at its maximum
    float2 ru;                             // R(u) of the winning bin
};

__device__ void fsr_block_mw(MwSmem &sm, const FsrArgs &a, int b)
{
    WarpSmem &ws = sm.ws;
    const Twiddles &tw = sm.tw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int status = *a.status;
    if (b == 0 && tid == 0 && a.status_out != nullptr) *a.status_out = status;
    if (status) return;
    const int H = a.H, W = a.W;
    const int nbx = (W + kFsrB - 1) / kFsrB, nby = (H + kFsrB - 1) / kFsrB;
    if (b >= nbx * nby) return;
    const int bi = b / nbx, bj = b - bi * nbx;
    const int o = (N - kFsrB) / 2;
    const int ys = kFsrB * bi - o, xs = kFsrB * bj - o;
    const FsrTables *tab = a.tab;

    // 1. support: warp w loads rows w, w + MW, ...
    for (int m = warp; m < N; m += MW) support_row(ws, a, m, xs + lane, ys + m, bi, bj, lane);
    __syncthreads();
    // 2. row DFTs: thread t < 2N transforms row t % N of the weights (t < N) or of the values
    {
        float x[N];
        const int row = tid & (N - 1);
        const float *src = tid < N ? ws.sup.w : ws.sup.f;
        if (tid < 2 * N) {
#pragma unroll
            for (int n = 0; n < N; ++n) x[n] = src[row * SS + n];
        }
        __syncthreads();                                   // the union is rewritten below
        if (tid < 2 * N) real_row_dft(x, &(tid < N ? ws.dft.w : ws.dft.f)[row * NH]);
    }
    __syncthreads();
    // 3. column DFTs in place: 17 columns of W, then 17 of R
    if (tid < 2 * NH) column_dft(tid < NH ? ws.dft.w : ws.dft.f, tid < NH ? tid : tid - NH);
    __syncthreads();

    // 4. this warp's slots of the half spectrum (layout as in fsr_block); warp 0 builds W
    const int k = lane;
    const bool upper = k > N / 2;
    const int kap = upper ? N - k : k;
    const int c0 = upper ? N / 2 : 0;
    const int rowbase = kap * N + c0;
    float2 Rr[MWS];
    float wfr[MWS];
#pragma unroll
    for (int j = 0; j < MWS; ++j) {
        const int sl = warp + MW * j;
        const bool mine = sl < NH;
        const int sc = mine ? sl : 0;
        const float2 r = ws.dft.f[k * NH + (upper ? NH - 1 - sc : sc)];
        Rr[j] = !mine ? make_float2(0.f, 0.f) : (upper ? make_float2(r.x, -r.y) : r);
        const bool held = mine && (!upper || (sc != 0 && sc != NH - 1));
        wfr[j] = held ? __ldg(&tab->wf[k * NH + (upper ? NH - 1 - sc : sc)]) : 0.f;
    }
    float2 Wt[NH];
    if (warp == 0) {
#pragma unroll
        for (int l = 0; l < NH; ++l) Wt[l] = ws.dft.w[k * NH + l];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int l = 0; l < NH; ++l) ws.W[k * WS + l] = Wt[l];
        __syncwarp();
#pragma unroll
        for (int l = NH; l < N; ++l) {
            const float2 w2 = ws.W[((N - k) & (N - 1)) * WS + (N - l)];
            ws.W[k * WS + l] = make_float2(w2.x, -w2.y);
        }
#pragma unroll
        for (int l = 0; l < NH; ++l) ws.W[k * WS + N + l] = ws.W[k * WS + l];
        if (lane < NH) ws.W[N * WS + lane] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float W0 = ws.W[0].x;

    const int pm = (lane >> 2) & 3, pn = lane & 3;
    const int jm = o + pm, jn = o + pn;
    float g = 0.f;
    const float gscale = W0 > 0.f ? a.gamma / W0 : 0.f;
    float gdr = 0.f, gdi = 0.f, gf = 0.f;
    int jp = 0;
    int it = 0;
    for (; it < a.iters && W0 > 0.f; ++it) {
        uint32_t key[MWS];
#pragma unroll
        for (int j = 0; j < MWS; ++j) {
            const float e = wfr[j] * fmaf(Rr[j].x, Rr[j].x, Rr[j].y * Rr[j].y);
            key[j] = (__float_as_uint(e) & ~31u) | (uint32_t)(31 - min(warp + MW * j, NH - 1));
        }
#pragma unroll
        for (int w = 1; w < MWS; w *= 2)
#pragma unroll
            for (int j = 0; j + w < MWS; j += 2 * w) key[j] = max(key[j], key[j + w]);
        const uint32_t best = key[0];
        const int cand = rowbase + 31 - (int)(best & 31);
        g = fmaf(gf, fmaf(gdr, tw.cs[jp], -gdi * tw.sn[jp]), g);
        gf = 0.f;
        const uint32_t mw = __reduce_max_sync(0xffffffffu, best);
        const int cw = __reduce_min_sync(0xffffffffu, ((best ^ mw) >> 5) == 0 ? cand : 0x7fffffff);
        if (lane == 0) {
            sm.redm[warp] = mw;
            sm.redc[warp] = cw;
        }
        __syncthreads();
        uint32_t m = 0;
#pragma unroll
        for (int w = 0; w < MW; ++w) m = max(m, sm.redm[w]);
        int win = 0x7fffffff;
#pragma unroll
        for (int w = 0; w < MW; ++w)
            if (((sm.redm[w] ^ m) >> 5) == 0) win = min(win, sm.redc[w]);
        if ((m >> 5) == 0) break;                        // residual exhausted (the whole block)
        if (a.sel != nullptr && tid == 0) a.sel[(size_t)b * a.iters + it] = (uint16_t)win;
        const int uk = win >> 5, ul = win & (N - 1);
        const int owner = ul <= N / 2 ? uk : N - uk;
        const int slot = ul <= N / 2 ? ul : ul - N / 2;
        if (warp == (slot & (MW - 1)) && lane == owner) {
            const int j = slot / MW;                       // warp-uniform
            float2 rv = Rr[0];
#pragma unroll
            for (int jj = 1; jj < MWS; ++jj) if (j == jj) rv = Rr[jj];
            sm.ru = rv;
        }
        __syncthreads();
        const float2 ru = sm.ru;
        const bool self = ((uk & (N / 2 - 1)) == 0) && ((ul & (N / 2 - 1)) == 0);
        const float dr = gscale * ru.x;
        const float di = self ? 0.f : gscale * ru.y;
        const float2 *pa = ws.W + ((kap - uk) & (N - 1)) * WS + ((c0 - ul) & (N - 1)) + warp;
        const float2 *pc = (self ? ws.W + N * WS
                                 : ws.W + ((kap + uk) & (N - 1)) * WS + ((c0 + ul) & (N - 1))) + warp;
        const float2 ndr = make_float2(-dr, -dr), ndi = make_float2(-di, -di);
#pragma unroll
        for (int j = 0; j < MWS; ++j) {
            if (warp + MW * j >= NH) break;                // slot 16: warp 0 only
            const float2 av = pa[MW * j], cv = pc[MW * j];
            const float2 sv = __fadd2_rn(av, cv);
            const float2 q = make_float2(cv.y - av.y, av.x - cv.x);
            Rr[j] = __ffma2_rn(ndi, q, __ffma2_rn(ndr, sv, Rr[j]));
        }
        jp = (uk * jm + ul * jn) & (N - 1);
        gdr = dr;
        gdi = di;
        gf = self ? 1.f : 2.f;
    }
    g = fmaf(gf, fmaf(gdr, tw.cs[jp], -gdi * tw.sn[jp]), g);
    if (a.sel != nullptr && warp == 0)                   // iterations not run: no selection
        for (int j = it + lane; j < a.iters; j += 32) a.sel[(size_t)b * a.iters + j] = 0xffffu;
    // 5. output: warp 0 holds the model at the 16 block pixels
    if (warp == 0 && lane < kFsrB * kFsrB) store_pixel(a, kFsrB * bi + pm, kFsrB * bj + pn, g);
}

__device__ __forceinline__ void load_twiddles(Twiddles &tw)
{
    if (threadIdx.x < N) {
        tw.cs[threadIdx.x] = c_cs[threadIdx.x];
        tw.sn[threadIdx.x] = c_sn[threadIdx.x];
    }
    __syncthreads();
}

// single-stream launch: one CTA = WPB1 consecutive blocks, one per warp
template <bool TRACE>
__global__ void __launch_bounds__(WPB1 * 32, 4) fsr_kernel(FrameTask t)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<WPB1> &sm = *reinterpret_cast<Smem<WPB1> *>(smem_raw);
    load_twiddles(sm.tw);
    const int warp = threadIdx.x >> 5;
    FsrArgs a;
    fsr_args(a, t);
    fsr_block<TRACE>(sm.tw, sm.w[warp], a, blockIdx.x * WPB1 + warp);
}

// Concealed weighting > 0: block (i, j) reads the blocks before it in raster order that overlap
// its support (rows i-4 .. i-1 at columns j-4 .. j+4, and row i left of j), so blocks run as
// wavefronts w = 5 i + j -- every such block has a smaller w.  One launch per wave; CTA b of the
// launch (MW warps) takes the b-th block (i = i_lo + b, j = w - 5 i) of that wave.
__global__ void __launch_bounds__(MW * 32) fsr_wave_kernel(FrameTask t, int wave, int i_lo, int count)
{
    __shared__ __align__(16) MwSmem sm;
    load_twiddles(sm.tw);
    const int b = blockIdx.x;
    if (b >= count) return;
    const int i = i_lo + b, j = wave - 5 * i;
    FsrArgs a;
    fsr_args(a, t);
    fsr_block_mw(sm, a, i * ((t.W + kFsrB - 1) / kFsrB) + j);
}

// batched form: CTAs claim tiles (WPB consecutive blocks of one task) in increasing order from
// the batch's tile queue, so each tile runs as in the single-stream launch (its warps start
// together on adjacent blocks and share their support rows in L1).  The next claim is issued
// before the current tile's work so that its latency is hidden.  Each warp keeps the arguments
// of its task in shared memory (refreshed when the task changes).
template <int WPB, bool TRACE>
__global__ void __launch_bounds__(WPB * 32, 16 / WPB) fsr_batched_kernel(BatchDesc *bd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<WPB> &sm = *reinterpret_cast<Smem<WPB> *>(smem_raw);
    int *queue = &bd->queue[kPhFsr];
    if (threadIdx.x == 0) sm.tile[0] = atomicAdd(queue, 1);
    load_twiddles(sm.tw);                              // ends with a barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = bd->ntiles[kPhFsr];
    int lo = 0, hi = -1;                               // tile range of the warp's cached task
    for (int it = 0;; ++it) {
        const int c = sm.tile[it & 1];
        if (c >= n) break;                             // uniform over the CTA
        int nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(queue, 1);
        if (c < lo || c >= hi) {                       // task change: refresh the warp's copy
            const int ti = batch_task(bd, kPhFsr, c);
            lo = bd->off[kPhFsr][ti];
            hi = bd->off[kPhFsr][ti + 1];
            __syncwarp();
            if (lane == 0) fsr_args(sm.args[warp], bd->task[ti]);
            __syncwarp();
        }
        fsr_block<TRACE>(sm.tw, sm.w[warp], sm.args[warp], (c - lo) * WPB + warp);
        // slot (it+1)&1 was last read before the previous barrier, so it may be rewritten now
        if (threadIdx.x == 0) sm.tile[(it + 1) & 1] = nxt;
        __syncthreads();
    }
}

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

namespace {
int g_ready[64];   // per device: constant twiddles and the shared-memory attribute are set
}

cudaError_t init_fsr(int dev)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_ready[dev]) return cudaSuccess;
    // DFT twiddles computed on the host (no device transcendental functions)
    float cs[N], sn[N];
    for (int j = 0; j < N; ++j) {
        cs[j] = (float)std::cos(2.0 * M_PI * j / N);
        sn[j] = (float)std::sin(2.0 * M_PI * j / N);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_cs, cs, sizeof(cs));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sn, sn, sizeof(sn));
    if (e == cudaSuccess) e = smem_attr(fsr_kernel<false>, sizeof(Smem<WPB1>));
    if (e == cudaSuccess) e = smem_attr(fsr_kernel<true>, sizeof(Smem<WPB1>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<2, false>, sizeof(Smem<2>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<4, false>, sizeof(Smem<4>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<8, false>, sizeof(Smem<8>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<2, true>, sizeof(Smem<2>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<4, true>, sizeof(Smem<4>));
    if (e == cudaSuccess) e = smem_attr(fsr_batched_kernel<8, true>, sizeof(Smem<8>));
    if (e == cudaSuccess) g_ready[dev] = 1;
    return e;
}

int tiles_fsr(const FrameTask &t, int fsr_blocks)
{
    const int nb = ((t.W + kFsrB - 1) / kFsrB) * ((t.H + kFsrB - 1) / kFsrB);
    return (nb + fsr_blocks - 1) / fsr_blocks;
}

namespace {
template <int WPB, bool TRACE>
void launch_fsr_batched_t(BatchDesc *bd, cudaStream_t st)
{
    static std::atomic<int> grids[64];
    const int grid = persistent_grid_cached(fsr_batched_kernel<WPB, TRACE>, WPB * 32, sizeof(Smem<WPB>), grids);
    fsr_batched_kernel<WPB, TRACE><<<grid, WPB * 32, sizeof(Smem<WPB>), st>>>(bd);
}

template <bool TRACE>
void launch_fsr_batched_b(BatchDesc *bd, int fsr_blocks, cudaStream_t st)
{
    switch (fsr_blocks) {
    case 2: launch_fsr_batched_t<2, TRACE>(bd, st); break;
    case 8: launch_fsr_batched_t<8, TRACE>(bd, st); break;
    default: launch_fsr_batched_t<4, TRACE>(bd, st); break;
    }
}
}  // namespace

cudaError_t launch_fsr_batched(BatchDesc *bd, int fsr_blocks, bool trace, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = init_fsr(dev);
    if (e != cudaSuccess) return e;
    if (trace) launch_fsr_batched_b<true>(bd, fsr_blocks, st);
    else launch_fsr_batched_b<false>(bd, fsr_blocks, st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fsr(const FrameTask &t, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = init_fsr(dev);
    if (e != cudaSuccess) return e;
    if (t.fsr_concealed > 0.f) {                       // wavefronts, one launch per wave
        const int nby = (t.H + kFsrB - 1) / kFsrB, nbx = (t.W + kFsrB - 1) / kFsrB;
        for (int w = 0; w <= 5 * (nby - 1) + nbx - 1; ++w) {
            const int i_lo = w - (nbx - 1) > 0 ? (w - (nbx - 1) + 4) / 5 : 0;
            const int i_hi = w / 5 < nby - 1 ? w / 5 : nby - 1;
            const int count = i_hi - i_lo + 1;
            if (count <= 0) continue;
            fsr_wave_kernel<<<count, MW * 32, 0, st>>>(t, w, i_lo, count);
            count_launch();
        }
        return cudaGetLastError();
    }
    if (t.fsr_sel != nullptr) fsr_kernel<true><<<tiles_fsr(t, WPB1), WPB1 * 32, sizeof(Smem<WPB1>), st>>>(t);
    else fsr_kernel<false><<<tiles_fsr(t, WPB1), WPB1 * 32, sizeof(Smem<WPB1>), st>>>(t);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
