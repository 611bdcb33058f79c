// ingest.cu -- takes the sensor data of frame t into the stream's ring slot.
//
// Quarter sampling (Sec. 1, Fig. 1): per 2x2 block exactly one pixel is measured; the sampled
// image is f_sub = f * b with the binary mask b (Sec. 2.1).  The kernel checks that the mask is a
// quarter-sampling mask (values 0/1, one 1 per block), writes the sample plane with unmeasured
// bytes zeroed and the mask as 0x00/0xFF bytes (the form the ME kernel ANDs with), and flags a
// bad mask in the frame status word so that the remaining kernels of the step do nothing.
#include <atomic>

#include "rfsr_internal.h"

namespace rfsr {

namespace {
std::atomic<long long> g_launches{0};
}

void count_launch(int n) { g_launches += n; }
long long launches() { return g_launches.load(); }

constexpr int kIngestThreads = 256;

int tiles_ingest(const FrameTask &t)
{
    const int nb = (t.H / 2) * (t.W / 2);
    return (nb + kIngestThreads - 1) / kIngestThreads;
}

__device__ __forceinline__ void ingest_tile(const FrameTask &t, int tile)
{
    const int bw = t.W >> 1, bh = t.H >> 1;
    const int i = tile * kIngestThreads + threadIdx.x;
    if (i == 0 && t.prev_status != nullptr && *t.prev_status != 0)
        atomicOr(t.status, kStatusPoisoned);
    if (i >= bw * bh) return;
    const int by = i / bw, bx = i - by * bw;
    const size_t o0 = (size_t)(2 * by) * t.W + 2 * bx, o1 = o0 + t.W;
    // two aligned 16-bit loads per plane (x is even)
    const uint16_t m0 = *reinterpret_cast<const uint16_t *>(t.in_msk + o0);
    const uint16_t m1 = *reinterpret_cast<const uint16_t *>(t.in_msk + o1);
    const uint16_t s0 = *reinterpret_cast<const uint16_t *>(t.in_smp + o0);
    const uint16_t s1 = *reinterpret_cast<const uint16_t *>(t.in_smp + o1);
    const int a = m0 & 0xff, b = m0 >> 8, c = m1 & 0xff, d = m1 >> 8;
    const bool ok = ((a | b | c | d) <= 1) && (a + b + c + d == 1);
    if (!ok) atomicOr(t.status, kStatusBadMask);
    // byte masks 0x00 / 0xff (an invalid byte still yields a well-formed plane)
    const uint16_t bm0 = (uint16_t)((a ? 0x00ff : 0) | (b ? 0xff00 : 0));
    const uint16_t bm1 = (uint16_t)((c ? 0x00ff : 0) | (d ? 0xff00 : 0));
    *reinterpret_cast<uint16_t *>(t.cur_msk + o0) = bm0;
    *reinterpret_cast<uint16_t *>(t.cur_msk + o1) = bm1;
    *reinterpret_cast<uint16_t *>(t.cur_smp + o0) = (uint16_t)(s0 & bm0);
    *reinterpret_cast<uint16_t *>(t.cur_smp + o1) = (uint16_t)(s1 & bm1);
}

__global__ void __launch_bounds__(kIngestThreads) ingest_kernel(FrameTask t)
{
    ingest_tile(t, blockIdx.x);
}

__global__ void __launch_bounds__(kIngestThreads) ingest_batched_kernel(BatchDesc *bd)
{
    __shared__ FrameTask task;
    __shared__ int claim[2];
    claim_tiles(bd, kPhIngest, task, claim, [](const FrameTask &t, int l) { ingest_tile(t, l); });
}

// start of a batched step: clear the status word of every task (ingest only ever sets bits)
__global__ void batch_prologue_kernel(BatchDesc *bd)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bd->ntasks; i += gridDim.x * blockDim.x)
        *bd->task[i].status = 0;
}

cudaError_t launch_batch_prologue(BatchDesc *bd, cudaStream_t st)
{
    batch_prologue_kernel<<<1, kMaxBatch, 0, st>>>(bd);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ingest(const FrameTask &t, cudaStream_t st)
{
    ingest_kernel<<<tiles_ingest(t), kIngestThreads, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ingest_batched(BatchDesc *bd, cudaStream_t st)
{
    static std::atomic<int> grids[64];
    const int grid = persistent_grid_cached(ingest_batched_kernel, kIngestThreads, 0, grids);
    ingest_batched_kernel<<<grid, kIngestThreads, 0, st>>>(bd);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
