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
// GB300 design: one warp per block.  R is Hermitian (the signal is real), so only the half
// spectrum l = 0..16 is kept: lane k holds R(k, 0..16) in registers.  The full weight spectrum W
// (needed at arbitrary shifts k -+ u) lives in shared memory with a padded row stride so that the
// 32 lanes' row-shifted reads are conflict-free.  The 2-D DFTs are row / column passes with a
// host-computed twiddle table (no device transcendental functions).  FP32 throughout.
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int N = kFsrN;
constexpr int NH = kFsrHalf;
constexpr int WPB = 4;                     // warps (blocks) per CTA
constexpr int WSTRIDE = N + 1;             // padded row stride of W (float2)

struct WarpSmem {
    float2 Wf[N * WSTRIDE];   // full weight spectrum; first holds the support (w, w*f)
    float2 rw[N * NH];        // row DFTs of the weights
    float2 rr[N * NH];        // row DFTs of the weighted values
};

struct Smem {
    float wsp[N * N];
    float wf[N * NH];
    float cs[N];
    float sn[N];
    WarpSmem w[WPB];
};

__global__ void __launch_bounds__(WPB * 32) fsr_kernel(FrameTask t)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FsrTables *tab = reinterpret_cast<const FsrTables *>(t.fsr_tables);
    for (int i = threadIdx.x; i < N * N; i += WPB * 32) sm.wsp[i] = tab->wsp[i];
    for (int i = threadIdx.x; i < N * NH; i += WPB * 32) sm.wf[i] = tab->wf[i];
    if (threadIdx.x < N) {
        sm.cs[threadIdx.x] = tab->cs[threadIdx.x];
        sm.sn[threadIdx.x] = tab->sn[threadIdx.x];
    }
    __syncthreads();
    if (*t.status) return;

    const int H = t.H, W = t.W;
    const int nbx = (W + kFsrB - 1) / kFsrB, nby = (H + kFsrB - 1) / kFsrB;
    const int b = blockIdx.x * WPB + warp;
    if (b >= nbx * nby) return;
    const int bi = b / nbx, bj = b - bi * nbx;
    const int o = (N - kFsrB) / 2;
    const int ys = kFsrB * bi - o, xs = kFsrB * bj - o;
    WarpSmem &ws = sm.w[warp];
    float *sw = reinterpret_cast<float *>(ws.Wf);           // support weights  [N][WSTRIDE]
    float *sf = sw + N * WSTRIDE;                           // weighted values [N][WSTRIDE]
    const float mu = t.fsr_proj_weight;

    // 1. support: lane = column, coalesced row loads
    for (int m = 0; m < N; ++m) {
        const int y = ys + m, x = xs + lane;
        float wt = 0.f, val = 0.f;
        if ((unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W) {
            const size_t i = (size_t)y * W + x;
            if (t.cur_msk[i]) {
                wt = sm.wsp[m * N + lane];
                val = (float)t.cur_smp[i] * (1.0f / 255.0f);
            } else if (t.pcnt != nullptr && t.pcnt[i]) {
                wt = mu * sm.wsp[m * N + lane];
                val = (float)t.psum[i] / (255.0f * (float)t.pcnt[i]);
            }
        }
        sw[m * WSTRIDE + lane] = wt;
        sf[m * WSTRIDE + lane] = wt * val;
    }
    __syncwarp();

    // 2. row DFTs (lane = row m): X(m, l) = sum_n a(m, n) exp(-2 pi i l n / N), l = 0..16
    {
        const int m = lane;
        for (int l = 0; l < NH; ++l) {
            float wr = 0.f, wi = 0.f, fr = 0.f, fi = 0.f;
#pragma unroll 8
            for (int n = 0; n < N; ++n) {
                const int j = (l * n) & (N - 1);
                const float c = sm.cs[j], s = sm.sn[j];
                const float a = sw[m * WSTRIDE + n], f = sf[m * WSTRIDE + n];
                wr = fmaf(a, c, wr);
                wi = fmaf(-a, s, wi);
                fr = fmaf(f, c, fr);
                fi = fmaf(-f, s, fi);
            }
            ws.rw[m * NH + l] = make_float2(wr, wi);
            ws.rr[m * NH + l] = make_float2(fr, fi);
        }
    }
    __syncwarp();

    // 3. column DFTs (lane = output row k); R stays in registers, W goes to shared memory
    float Rre[NH], Rim[NH];
    const int k = lane;
#pragma unroll
    for (int l = 0; l < NH; ++l) {
        float wr = 0.f, wi = 0.f, fr = 0.f, fi = 0.f;
        for (int m = 0; m < N; ++m) {
            const int j = (k * m) & (N - 1);
            const float c = sm.cs[j], s = -sm.sn[j];        // exp(-i a) = c + i s
            const float2 a = ws.rw[m * NH + l], f = ws.rr[m * NH + l];
            wr = fmaf(a.x, c, fmaf(-a.y, s, wr));
            wi = fmaf(a.x, s, fmaf(a.y, c, wi));
            fr = fmaf(f.x, c, fmaf(-f.y, s, fr));
            fi = fmaf(f.x, s, fmaf(f.y, c, fi));
        }
        ws.Wf[k * WSTRIDE + l] = make_float2(wr, wi);
        Rre[l] = fr;
        Rim[l] = fi;
    }
    __syncwarp();
    // W(k, l) for l = 17..31 from Hermitian symmetry: W(k, l) = conj(W(-k, -l))
    for (int l = NH; l < N; ++l) {
        const float2 a = ws.Wf[((N - k) & (N - 1)) * WSTRIDE + (N - l)];
        ws.Wf[k * WSTRIDE + l] = make_float2(a.x, -a.y);
    }
    __syncwarp();
    const float W0 = ws.Wf[0].x;

    // block pixel owned by lanes 0..15
    const int pm = (lane >> 2) & 3, pn = lane & 3;
    float g = 0.f;

    // 4. iterations
    const float gamma = t.fsr_gamma;
    for (int it = 0; it < t.fsr_iters && W0 > 0.f; ++it) {
        float be = -1.f, bre = 0.f, bim = 0.f;
        int bkey = 0x7fffffff, bu = 0;
#pragma unroll
        for (int l = 0; l < NH; ++l) {
            const bool canon = (l != 0 && l != NH - 1) || k <= N / 2;
            const float e = sm.wf[k * NH + l] * fmaf(Rre[l], Rre[l], Rim[l] * Rim[l]);
            const int lin = k * N + l;
            const int clin = ((N - k) & (N - 1)) * N + ((N - l) & (N - 1));
            const int key = min(lin, clin);
            if (canon && (e > be || (e == be && key < bkey))) {
                be = e; bkey = key; bu = lin; bre = Rre[l]; bim = Rim[l];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oe = __shfl_xor_sync(0xffffffffu, be, off);
            const int ok = __shfl_xor_sync(0xffffffffu, bkey, off);
            const int ou = __shfl_xor_sync(0xffffffffu, bu, off);
            if (oe > be || (oe == be && ok < bkey)) {
                be = oe; bkey = ok; bu = ou;
            }
        }
        const int src = bu >> 5;
        const float ure = __shfl_sync(0xffffffffu, bre, src);
        const float uim = __shfl_sync(0xffffffffu, bim, src);
        if (!(be > 0.f)) break;                              // residual exhausted
        const int uk = bu >> 5, ul = bu & (N - 1);
        const bool self = ((uk & (N / 2 - 1)) == 0) && ((ul & (N / 2 - 1)) == 0);
        const float dr = gamma * ure / W0;
        const float di = self ? 0.f : gamma * uim / W0;
        // residual update over the half spectrum held by this lane
        const int ra = ((k - uk) & (N - 1)) * WSTRIDE, rb = ((k + uk) & (N - 1)) * WSTRIDE;
        if (self) {
#pragma unroll
            for (int l = 0; l < NH; ++l) {
                const float2 a = ws.Wf[ra + ((l - ul) & (N - 1))];
                Rre[l] = fmaf(-dr, a.x, Rre[l]);
                Rim[l] = fmaf(-dr, a.y, Rim[l]);
            }
        } else {
#pragma unroll
            for (int l = 0; l < NH; ++l) {
                const float2 a = ws.Wf[ra + ((l - ul) & (N - 1))];
                const float2 c = ws.Wf[rb + ((l + ul) & (N - 1))];
                // dc * a + conj(dc) * c
                const float xr = dr * (a.x + c.x) + di * (c.y - a.y);
                const float xi = dr * (a.y + c.y) + di * (a.x - c.x);
                Rre[l] -= xr;
                Rim[l] -= xi;
            }
        }
        // model at the block pixel of this lane: g += (1 or 2) Re(dc phi_u)
        const int j = (uk * (o + pm) + ul * (o + pn)) & (N - 1);
        const float re_part = dr * sm.cs[j] - di * sm.sn[j];
        g += self ? re_part : 2.f * re_part;
    }

    // 5. output: D-FSR overwrite and the 8-bit reconstruction
    if (lane < kFsrB * kFsrB) {
        const int y = kFsrB * bi + pm, x = kFsrB * bj + pn;
        if (y < H && x < W) {
            const size_t i = (size_t)y * W + x;
            float v = g;
            uint8_t q;
            if (t.cur_msk[i]) {
                v = (float)t.cur_smp[i] * (1.0f / 255.0f);
                q = t.cur_smp[i];
            } else {
                if (t.fsr_overwrite_projected && t.pcnt != nullptr && t.pcnt[i])
                    v = (float)t.psum[i] / (255.0f * (float)t.pcnt[i]);
                const float r = rintf(255.0f * v);
                q = (uint8_t)fminf(fmaxf(r, 0.0f), 255.0f);
            }
            if (t.fsr_out) t.fsr_out[i] = v;
            if (t.cur_rec) t.cur_rec[i] = q;
            if (t.out_u8) t.out_u8[i] = q;
        }
    }
}

}  // namespace

cudaError_t launch_fsr(const FrameTask &t, cudaStream_t st)
{
    static bool attr_set = false;
    const size_t smem = sizeof(Smem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fsr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int nb = ((t.W + kFsrB - 1) / kFsrB) * ((t.H + kFsrB - 1) / kFsrB);
    fsr_kernel<<<(nb + WPB - 1) / WPB, WPB * 32, smem, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
