// rfsr_internal.h -- device data layout and kernel launchers shared by the library's CUDA
// translation units.  Not part of the public ABI (include/rfsr.h is).
#pragma once

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

// One frame step of one stream: every pointer is device memory owned by the stream, except
// in_smp / in_msk which point at the staged (or caller's device) input.
struct FrameTask {
    int H, W;
    int K;              // references actually used for this frame (0..kMaxRefs)
    int T, R, Rc;
    int cc_mode;
    // FSR
    int fsr_iters;
    float fsr_gamma;
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
};

// A batched frame step: up to kMaxBatch frame tasks (one per stream) run by one persistent
// launch per phase.  Each phase flattens its tiles over the tasks: task i owns the tiles
// [off[phase][i], off[phase][i+1]) and a CTA finds the task of a tile by binary search.
constexpr int kMaxBatch = 256;
enum Phase { kPhIngest = 0, kPhMe = 1, kPhRme = 2, kPhCc = 3, kPhFsr = 4, kPhases = 5 };

struct BatchDesc {
    int ntasks;
    int ntiles[kPhases];
    int queue[kPhases];                    // tile queue heads (0 in the host copy; atomic claims)
    int off[kPhases][kMaxBatch + 1];
    FrameTask task[kMaxBatch];
};

// tiles of a task in each phase (the single-stream launches use the same decomposition)
int tiles_ingest(const FrameTask &t);
int tiles_me(const FrameTask &t);
int tiles_rme(const FrameTask &t);
int tiles_cc(const FrameTask &t);
int tiles_fsr(const FrameTask &t);         // CTAs of WPB blocks (single-stream launch)

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

// batched launchers: one persistent launch per phase over all tasks of bd (device pointer);
// the grid sizes depend only on the device, so the sequence can be captured in a CUDA graph
cudaError_t launch_batch_prologue(const BatchDesc *bd, cudaStream_t st);
cudaError_t launch_ingest_batched(const BatchDesc *bd, cudaStream_t st);
cudaError_t launch_me_batched(const BatchDesc *bd, int T, cudaStream_t st);
cudaError_t launch_rme_batched(const BatchDesc *bd, cudaStream_t st);
cudaError_t launch_cc_batched(const BatchDesc *bd, int T, cudaStream_t st);
cudaError_t launch_fsr_batched(const BatchDesc *bd, cudaStream_t st);

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
cudaError_t launch_fsr(const FrameTask &t, cudaStream_t st);
// one-time per-device set-up of the FSR kernel (constant twiddles, shared-memory limit)
cudaError_t init_fsr(int device);

// set the calling thread's rfsr_last_error() message; returns code
int set_error(int code, const std::string &msg);

// number of kernel launches issued by this process (all launchers count)
void count_launch(int n = 1);
long long launches();

}  // namespace rfsr
