// rfsr_internal.h -- device data layout and kernel launchers shared by the library's CUDA
// translation units.  Not part of the public ABI (include/rfsr.h is).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace rfsr {

constexpr int kMaxRefs = 3;        // K (Sec. 4 uses three previous frames)
constexpr int kMaxHalf = 5;        // template half size h = T/2, T <= 11
constexpr int kMaxRadius = 9;      // search radius R <= 9 (Sec. 3.1.1 uses {-9..9})
constexpr int kFsrN = 32;          // FSR support / DFT size
constexpr int kFsrB = 4;           // FSR block size
constexpr int kFsrHalf = kFsrN / 2 + 1;   // stored half spectrum: l = 0..16

// device status bits (per frame, written by kernels, read back by the host)
constexpr int kStatusBadMask = 1;     // this frame's mask is not a quarter-sampling mask
constexpr int kStatusPoisoned = 2;    // an earlier frame of the stream had a bad mask
constexpr int kStatusWaitTimeout = 4; // a wait of the fused ME + checks launch ran out

// One frame step of one stream: every pointer is device memory owned by the stream, except
// in_smp / in_msk which point at the staged (or caller's device) input.
struct FrameTask {
    int H, W;
    int K;              // references actually used for this frame (0..kMaxRefs)
    int T, R, Rc;
    int me_pred;        // predictive-centre window radius for references 2..K (0: full search)
    int cc_mode;
    // FSR
    int fsr_iters;
    float fsr_gamma;
    float fsr_concealed;       // concealed weighting delta (0: blocks independent)
    float fsr_proj_weight;
    int fsr_overwrite_projected;
    const float *fsr_tables;   // FsrTables in device memory
    // input
    const uint8_t *in_smp;
    const uint8_t *in_msk;     // 0/1 bytes
    // ring slot of frame t: sample plane (samples & mask), byte mask 0x00/0xFF, reconstruction
    uint8_t *cur_smp;
    uint8_t *cur_msk;
    uint8_t *cur_rec;
    // ring slots of frames t-1..t-K
    const uint8_t *ref_rec[kMaxRefs];
    const uint8_t *ref_smp[kMaxRefs];
    const uint8_t *ref_msk[kMaxRefs];
    // per-reference planes
    int8_t *mv[kMaxRefs];      // raw ME field, 2 x int8 per pixel
    int8_t *fmv[kMaxRefs];     // vector used by checks / projection
    uint8_t *dec[kMaxRefs];    // decision labels
    int8_t *rmv[kMaxRefs];     // reverse field at every past-frame pixel (RME mode)
    // projection and FSR
    uint16_t *psum;
    uint8_t *pcnt;
    float *fsr_out;            // FSR output of this frame, [0, 1] scale
    uint8_t *out_u8;           // optional extra copy of the reconstruction (per in-flight slot)
    int *status;               // frame status word (kStatus* bits)
    const int *prev_status;    // status word of the previous frame of the stream (poison chain)
    int *status_out;           // optional: receives the final status word (written by FSR)
    uint16_t *fsr_sel;         // optional: selected basis pair per block and iteration (trace)
};

// A batched frame step: up to kMaxBatch frame tasks (one per stream) run by one persistent
// launch per phase.  Each phase flattens its tiles over the tasks: task i owns the tiles
// [off[phase][i], off[phase][i+1]).  The tiles of a phase form a queue: CTAs claim them in
// increasing order with an atomic on the phase's queue head and find the task of a tile by binary
// search over the offsets.
constexpr int kMaxBatch = 256;
enum Phase { kPhIngest = 0, kPhMe = 1, kPhRme = 2, kPhCc = 3, kPhFsr = 4, kPhases = 5 };

struct BatchDesc {
    int ntasks;
    int ntiles[kPhases];
    int queue[kPhases];                    // tile queue heads (0 in the host copy; atomic claims)
    int off[kPhases][kMaxBatch + 1];
    FrameTask task[kMaxBatch];
};

// Tile shapes of the batched launches.  Every shape computes bit-identical results; they differ
// only in how the work is cut, so the engine may choose among them by measurement.
struct BatchShape {
    int me_warps = 8;                      // ME (T = 9): 8-row warp strips stacked per CTA (4 | 8)
    int me_box = 0;                        // ME (T = 9): 1 = the sliding-window box-sum kernel
    int fsr_blocks = 4;                    // FSR: 4x4 blocks (one per warp) per CTA (2 | 4 | 8)
};
bool shape_valid(const BatchShape &s);

// tiles of a task in each phase (the single-stream launches use the default shape)
int tiles_ingest(const FrameTask &t);
int tiles_me(const FrameTask &t, int me_warps = 8, int me_box = 0);
int tiles_rme(const FrameTask &t);
int tiles_cc(const FrameTask &t);
int tiles_fsr(const FrameTask &t, int fsr_blocks = 4);

// task of flattened tile `tile` of phase ph (binary search over the offsets)
__device__ __forceinline__ int batch_task(const BatchDesc *bd, int ph, int tile)
{
    int lo = 0, hi = bd->ntasks;           // off[ph][lo] <= tile < off[ph][hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bd->off[ph][mid] <= tile) lo = mid;
        else hi = mid;
    }
    return lo;
}

// copy a task into shared memory (all threads of the CTA call it; ends with a barrier)
__device__ __forceinline__ void load_task(FrameTask &dst, const FrameTask &src)
{
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(FrameTask) / sizeof(int)); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// The claim loop of a CTA-granular batched kernel (all threads of the CTA call it): tiles of
// phase ph are claimed from the queue in increasing order, the next claim is issued before the
// current tile's work (its latency overlaps the work), the tile's task is copied to shared memory
// when it changes, and fn(task, tile index within the task) runs once per claimed tile.  claim is
// a 2-int shared buffer; a barrier separates consecutive tiles.
template <typename Fn>
__device__ __forceinline__ void claim_tiles(BatchDesc *bd, int ph, FrameTask &task, int *claim, Fn &&fn)
{
    int *queue = &bd->queue[ph];
    const int n = bd->ntiles[ph];
    if (threadIdx.x == 0) claim[0] = atomicAdd(queue, 1);
    __syncthreads();
    int cached = -1;
    for (int it = 0;; ++it) {
        const int c = claim[it & 1];
        if (c >= n) break;                             // uniform over the CTA
        int nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(queue, 1);
        const int ti = batch_task(bd, ph, c);
        if (ti != cached) {
            load_task(task, bd->task[ti]);             // the previous tile ended with a barrier
            cached = ti;
        }
        fn(static_cast<const FrameTask &>(task), c - bd->off[ph][ti]);
        // slot (it+1)&1 was last read before the previous barrier, so it may be rewritten now
        if (threadIdx.x == 0) claim[(it + 1) & 1] = nxt;
        __syncthreads();
    }
}

// Resident CTAs per SM x SMs for a batched kernel (its persistent grid).
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1)
        per = 1;
    return sms * per;
}

// The persistent grid of a batched kernel on the calling thread's current device, computed once
// per device and call site (cache: one slot per device ordinal, 0 = not computed yet), so that an
// engine on another device gets its own device's figure.
template <typename K>
int persistent_grid_cached(K kernel, int threads, size_t smem, std::atomic<int> (&cache)[64])
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return persistent_grid(kernel, threads, smem);
    int g = cache[dev].load();
    if (g <= 0) {
        g = persistent_grid(kernel, threads, smem);
        cache[dev].store(g);
    }
    return g;
}

// batched launchers: one persistent launch per phase over all tasks of bd (device pointer; the
// kernels advance its queue heads); the grid sizes depend only on the device and the shape, so
// the sequence can be captured in a CUDA graph
cudaError_t launch_batch_prologue(BatchDesc *bd, cudaStream_t st);
cudaError_t launch_ingest_batched(BatchDesc *bd, cudaStream_t st);
cudaError_t launch_me_batched(BatchDesc *bd, int T, int me_warps, int me_box, cudaStream_t st);
cudaError_t launch_rme_batched(BatchDesc *bd, int T, cudaStream_t st);
// RME reverse field for T = 9 (tiled; other T use the direct search of cc.cu)
int tiles_rme9(const FrameTask &t);
cudaError_t launch_rme9(const FrameTask &t, cudaStream_t st);
cudaError_t launch_rme9_batched(BatchDesc *bd, cudaStream_t st);
cudaError_t launch_cc_batched(BatchDesc *bd, int T, cudaStream_t st);
// trace: run the instantiation that records FSR selections of the tasks that ask for them
cudaError_t launch_fsr_batched(BatchDesc *bd, int fsr_blocks, bool trace, cudaStream_t st);

// FSR tables computed on the host (no device transcendentals): spatial weights rho^d over the
// support, frequency weights over the stored half spectrum and the DFT twiddles.
struct FsrTables {
    float wsp[kFsrN * kFsrN];
    float wf[kFsrN * kFsrHalf];
    float cs[kFsrN];
    float sn[kFsrN];
};

// kernel launchers (each returns the CUDA error of the launch)
cudaError_t launch_ingest(const FrameTask &t, cudaStream_t st);
cudaError_t launch_me(const FrameTask &t, cudaStream_t st);
cudaError_t launch_rme_field(const FrameTask &t, cudaStream_t st);
cudaError_t launch_cc_project(const FrameTask &t, cudaStream_t st);

// Fused ME + checks + projection of one frame (T = 9, no RME, full ME search): one persistent
// launch whose CTAs claim, in order, ME tiles (64-row strips x 120 columns x past frame) and check
// tiles (32 x 32); a check tile first waits for the ME bands it reads.  The order is built on the
// host so that every tile's dependencies come earlier in it.
struct MeccPlan {
    const uint32_t *items;     // the frame's tiles in claim order (device)
    int nitems;
    int *ctr;                  // [0] claim head, [1] wait ran out, [2 + b] finished ME tiles of band b,
                               // [2 + nbands] a status word that stays 0 (the tiles' t.status, so
                               // that every thread of a CTA reads the same); zeroed before the launch
    int *status;               // the frame's status word (the ingest's verdict; a wait that runs out
                               // adds kStatusWaitTimeout)
    int nbands;                // 64-row ME bands
    int need;                  // ME tiles per band (column tiles x past frames)
    int limit;                 // polls of a wait before it gives up
    int bias;                  // 0; 1 makes every wait run out (tests of the timeout path)
};
// items of the claim order for an H x W frame with K past frames on a grid of `grid` CTAs
// (written to `items` unless null; returns the count)
int mecc_schedule(int H, int W, int K, int grid, uint32_t *items);
int mecc_bands(int H);
int mecc_need(int W, int K);
int mecc_grid();               // the fused kernel's persistent grid on the current device
cudaError_t launch_me_cc(const FrameTask &t, const MeccPlan &plan, cudaStream_t st);
cudaError_t launch_fsr(const FrameTask &t, cudaStream_t st);
// one-time per-device set-up of the FSR kernel (constant twiddles, shared-memory limit)
cudaError_t init_fsr(int device);
// one-time per-device set-up of the check kernel (reverse-check lane orders)
cudaError_t init_cc(int device);
// one-time per-device set-up of the T = 9 ME kernels (shared-memory limit)
cudaError_t init_me(int device);

// set the calling thread's rfsr_last_error() message; returns code
int set_error(int code, const std::string &msg);

// number of kernel launches issued by this process (all launchers count)
void count_launch(int n = 1);
long long launches();

}  // namespace rfsr
