// alu_peaks.cu -- throughput probes for the roofline denominators of the integer (ME, checks)
// and FP32 (FSR) kernels: long chains of one instruction kind, eight independent chains per
// thread, enough warps to fill every SM.  The result is instructions per clock per SM (from
// clock64 on the device) and per second (from CUDA events), for the kinds the kernels use.
#include <cstdint>

#include "rfsr.h"
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

template <int OP>
__device__ __forceinline__ uint32_t op(uint32_t a, uint32_t b, uint32_t c)
{
    if constexpr (OP == 0) return a + b + c;                          // 3-input add
    else if constexpr (OP == 1) return (a & b) ^ (~a & c);            // 3-input logic
    else if constexpr (OP == 2) return __byte_perm(a, b, 0x5140);     // byte permute
    else if constexpr (OP == 3) return __vabsdiffu4(a, b);            // byte |a-b|
    else if constexpr (OP == 4) return __vsadu4(a, b) + c;            // byte SAD (+ add)
    else if constexpr (OP == 5) return __vimax3_u16x2(a, b, c);       // 16-bit x2 3-way max
    else if constexpr (OP == 6) return __vimin3_u16x2(a, b, c);       // 16-bit x2 3-way min
    else if constexpr (OP == 7) return a * b + c;                     // integer multiply-add
    else if constexpr (OP == 8) return __sad(a, b, c);                // |a-b| + c
    else if constexpr (OP == 9) return min(a, b);                     // 32-bit min
    else return a ^ b;
}

// kind 12: the chains alternate between a 3-input add and an integer multiply-add, the mix of an
// integer kernel that spreads its additions over both pipes
// kind 13: byte SAD with its accumulate as one SIMD-video instruction
__device__ __forceinline__ uint32_t sad4_acc(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// kind 14: signed 16-bit x2 minimum; kind 15: sum of the two signed 16-bit |a-b| plus c (the L1
// distance of two packed vectors) as one SIMD-video instruction
__device__ __forceinline__ uint32_t min_s16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t sad2_acc(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("vabsdiff2.s32.s32.s32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int OP>
__device__ __forceinline__ uint32_t op_chain(int i, uint32_t a, uint32_t b, uint32_t c)
{
    if constexpr (OP == 12) return (i & 1) ? a * b + c : a + b + c;
    else if constexpr (OP == 13) return sad4_acc(a, b, c);
    else if constexpr (OP == 14) return min_s16x2(a, b);
    else if constexpr (OP == 15) return sad2_acc(a, b, c);
    else if constexpr (OP == 16) return (uint32_t)__vimax3_s16x2((int)a, (int)b, (int)c);
    else if constexpr (OP == 17) return __vimax3_u32(a, b, c);
    else return op<OP>(a, b, c);
}

template <int OP>
__global__ void __launch_bounds__(256) int_kernel(uint32_t *out, long long *cycles, int iters,
                                                 uint32_t seed)
{
    uint32_t v[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) v[i] = seed * (threadIdx.x + 1) + i * 0x9e3779b9u;
    const uint32_t c = seed ^ 0x5bd1e995u;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) v[i] = op_chain<OP>(i, v[i], v[(i + 1) % CHAINS], c);
    }
    const long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = x;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(256) ffma_kernel(uint32_t *out, long long *cycles, int iters,
                                                  uint32_t seed)
{
    float v[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) v[i] = (float)(seed + threadIdx.x + i) * 1e-3f;
    const float c = 0.999f;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) v[i] = fmaf(v[i], c, v[(i + 1) % CHAINS]);
    }
    const long long t1 = clock64();
    float x = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) x += v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = __float_as_uint(x);
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <typename K>
cudaError_t run(K kernel, int sms, int iters, double *ops_per_sec, double *ops_per_clk_sm)
{
    const int blocks = sms * 8, threads = 256;
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaMalloc(&out, sizeof(uint32_t) * blocks * threads);
    if (err) return err;
    err = cudaMalloc(&cyc, sizeof(long long) * blocks);
    if (err) { cudaFree(out); return err; }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kernel<<<blocks, threads>>>(out, cyc, 4, 12345u);          // warm-up
    cudaEventRecord(e0);
    kernel<<<blocks, threads>>>(out, cyc, iters, 12345u);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long *hc = new long long[blocks];
    cudaMemcpy(hc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    long long mx = 0;
    for (int i = 0; i < blocks; ++i) mx = hc[i] > mx ? hc[i] : mx;
    delete[] hc;
    const double ops = (double)blocks * threads * iters * UNROLL * CHAINS;
    *ops_per_sec = ops / (ms * 1e-3);
    // blocks of one SM run concurrently (8 x 256 threads fit), so per-SM ops over the slowest
    // block's cycle count is the per-SM rate
    *ops_per_clk_sm = (ops / sms) / (double)mx;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    count_launch(2);
    return err ? err : cudaGetLastError();
}

}  // namespace

}  // namespace rfsr

extern "C" int rfsr_alu_peak(int device, int kind, int iters, double *ops_per_sec,
                             double *ops_per_clk_sm)
{
    using namespace rfsr;
    if (!ops_per_sec || !ops_per_clk_sm || iters <= 0 || kind < 0 || kind > 17)
        return RFSR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return RFSR_EDEVICE;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return RFSR_EDEVICE;
    cudaError_t e;
    switch (kind) {
    case 0: e = run(int_kernel<0>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 1: e = run(int_kernel<1>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 2: e = run(int_kernel<2>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 3: e = run(int_kernel<3>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 4: e = run(int_kernel<4>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 5: e = run(int_kernel<5>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 6: e = run(int_kernel<6>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 7: e = run(int_kernel<7>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 8: e = run(int_kernel<8>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 12: e = run(int_kernel<12>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 13: e = run(int_kernel<13>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 14: e = run(int_kernel<14>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 15: e = run(int_kernel<15>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 16: e = run(int_kernel<16>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 17: e = run(int_kernel<17>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 9: e = run(int_kernel<9>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    case 10: e = run(int_kernel<10>, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    default: e = run(ffma_kernel, sms, iters, ops_per_sec, ops_per_clk_sm); break;
    }
    return e == cudaSuccess ? RFSR_OK : RFSR_EDEVICE;
}
