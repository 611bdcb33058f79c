/*
 * rfsr.h -- C ABI of the GB300 library for recursive frequency-selective reconstruction (R-FSR)
 * of quarter-sampled video (Grosche, Seiler, Kaup, ICIP 2021, arXiv 2203.09200).
 *
 * Per frame t of a stream the library runs, on the GPU and without a host round trip
 * (the processing chain of Fig. 1):
 *   ingest ... the sensor data: one measured pixel per 2x2 block (quarter sampling, Sec. 1) as a
 *              sample plane f_sub = f * b and a binary mask b (Sec. 2.1)
 *   ME ....... pixel-wise template matching of the measured pixels of frame t against each of the
 *              K previously reconstructed frames (Sec. 2.2; K = 3, Sec. 4)
 *   CC ....... consistency checks of the motion vectors: RME (Sec. 2.2), RMC / FRMC (Sec. 3.1.1),
 *              NNC (Sec. 3.1.2, Eq. (1)) and the proposed NNC + FRMC combination
 *   PR ....... projection of measured past pixels along accepted vectors, averaged over the
 *              past frames that project (Sec. 2.2)
 *   FSR ...... block-wise frequency selective reconstruction with the projected pixels as extra
 *              known pixels and the D-FSR overwrite rule (Sec. 2.1, 3.2), concealed weighting 0
 *              so all blocks are independent (Sec. 4)
 * and keeps the 8-bit reconstruction as the reference of the next frames.
 *
 * Conventions shared by all calls:
 *   - frames are H x W row-major 8-bit luma, H and W even, 16 <= H, W <= 8192;
 *   - a mask is H x W bytes, 1 = measured, 0 = not measured, with exactly one 1 per 2x2 block;
 *   - a motion vector is two int8 (vertical, horizontal) per pixel; it points from the current
 *     frame t into the past frame t-k;
 *   - every call returns RFSR_OK (0) or a negative RFSR_E* code; rfsr_last_error() gives a
 *     message for the calling thread; no C++ exception crosses this interface;
 *   - the engine is thread-safe; one stream must be used by one thread at a time;
 *   - device pointers are CUDA device addresses on the engine's device; host pointers are plain
 *     process memory.  The library never takes ownership of caller buffers.
 */
#ifndef RFSR_H
#define RFSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RFSR_ABI_VERSION 1

/* ---- status codes ---------------------------------------------------------------------- */
enum {
    RFSR_OK = 0,
    RFSR_EINVAL = -1,     /* bad argument: NULL pointer, size, parameter out of range       */
    RFSR_EMASK = -2,      /* mask is not a quarter-sampling mask (one 1 per 2x2, values 0/1) */
    RFSR_ENOMEM = -3,     /* device or pinned host memory could not be allocated            */
    RFSR_EAGAIN = -4,     /* stream queued by memory admission, not live yet                */
    RFSR_EBUSY = -5,      /* in-flight frame limit reached: collect frames first            */
    RFSR_ETIMEDOUT = -6,  /* nothing ready within the timeout                               */
    RFSR_EDEVICE = -7,    /* CUDA error; the message names the call                         */
    RFSR_ESTATE = -8      /* call not valid in the current state (e.g. get before push)     */
};

/* ---- consistency-check modes (Table 3 rows, plus no check and NNC alone) ---------------- */
enum {
    RFSR_CC_NONE = 0,      /* every projectable vector accepted                              */
    RFSR_CC_RME = 1,       /* reverse motion estimation, accept iff vectors coincide (Sec. 2.2) */
    RFSR_CC_RMC = 2,       /* reverse motion check, (2Rc+1)^2 reverse vectors (Sec. 3.1.1)   */
    RFSR_CC_FRMC = 3,      /* fast RMC, offsets {-7,-3,-1,0,1,3,7}^2 (Sec. 3.1.1)           */
    RFSR_CC_NNC = 4,       /* nearest neighbour check alone (Sec. 3.1.2)                     */
    RFSR_CC_NNC_FRMC = 5   /* NNC, then FRMC for NNC survivors: the paper's proposal         */
};

/* ---- per-pixel decision labels (debug plane RFSR_DBG_DECISION) -------------------------- */
enum {
    RFSR_DEC_MEASURED = 0,         /* pixel measured in frame t: nothing to project          */
    RFSR_DEC_NOT_PROJECTABLE = 1,  /* p+v outside the frame or not measured in frame t-k    */
    RFSR_DEC_NNC_REJECT = 2,       /* rejected by the nearest neighbour check               */
    RFSR_DEC_CHECK_REJECT = 3,     /* rejected by RME / RMC / FRMC                           */
    RFSR_DEC_ACCEPT = 4            /* projected                                              */
};

enum { RFSR_MASK_FIXED = 0, RFSR_MASK_DYNAMIC = 1 };

/* ---- configuration ---------------------------------------------------------------------- */
typedef struct rfsr_engine rfsr_engine;
typedef struct rfsr_stream rfsr_stream;

typedef struct {
    int device;            /* CUDA device ordinal                                                */
    size_t memory_budget;  /* bytes of device memory for stream state; 0 = 80% of free memory    */
    void *cuda_stream;     /* cudaStream_t to run on; NULL = the engine creates its own          */
    int max_inflight;      /* frames per stream pushed and not yet collected; 0 = 4             */
    int batched;           /* 0: each push launches its frame step at once; 1: pushes are staged
                              and rfsr_engine_step() runs one batched step over all streams      */
    int profile;           /* 1: record CUDA events between the phases of every frame step
                              (rfsr_stream_phase_ms) or around every batched step
                              (rfsr_engine_last_step_ms)                                         */
    int serve;             /* 1: batched engine with its own thread that launches a batched step
                              whenever frames are staged (continuous batching); implies batched  */
    int autotune;          /* batched engines, 1 (default): the first batched steps measure the
                              tile shapes (rfsr_batch_shape) and keep the fastest; 0: default
                              shape.  Results are identical for every shape.                    */
    /* Optional device allocator for the engine's device memory (stream state, batch tables), for
     * a caller that manages GPU memory itself (e.g. a framework's caching allocator).  NULL:
     * cudaMalloc / cudaFree.  Set both or neither.  dev_alloc returns NULL on failure (ENOMEM);
     * memory is released with dev_free only after every frame that used it has finished. */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;       /* passed to both callbacks                                          */
    int fuse_me_cc;        /* 0 (default): ME and the checks + projection are separate launches.
                              1: an unbatched stream with T = 9, the full ME search and a check
                              mode other than RME runs them as one persistent launch whose check
                              tiles wait (bounded) for the ME bands they read; same results, its
                              phase timing reports ME and checks together.  Measured slower at
                              1080p (1.23 against 1.13 ms), so it is off by default.            */
    int wait_test;         /* tests only, leave 0.  1: every wait of the fused launch runs out
                              (a count no ME tile reaches, a short limit), so the frame ends with
                              EDEVICE from rfsr_get_frame and the context stays usable.          */
} rfsr_engine_config;

/* Tile shapes of the batched launches (a performance choice only; no counterpart in the paper,
 * every shape gives bit-identical results). */
typedef struct {
    int me_tile_rows;      /* ME (T = 9) template tile of a CTA: 32 or 64 rows x 120 columns; the
                              staged search window is the tile + (T - 1) + 2R rows (default 64)  */
    int fsr_blocks;        /* FSR 4x4 blocks per CTA (one per warp): 2, 4 or 8 (default 4)        */
    int me_variant;        /* ME algorithm for T = 9: 0 warp-strip byte SIMD (default), 1 sliding-
                              window box sums over 32x64 tiles (same vectors: both are the exact
                              argmin with the same tie order)                                    */
} rfsr_batch_shape;

/* State of a batched engine's autotuner (rfsr_engine_get_tuning). */
typedef struct {
    int tuned;                 /* 1: the shape is final (measured, set, or tuning off)            */
    int steps;                 /* tuning steps measured so far                                    */
    rfsr_batch_shape shape;    /* the shape the batched steps use now                             */
    float me_ns[3];            /* mean device ns per pixel x reference: strips of 64 rows, strips of
                                  32 rows, box sums (0: not measured)                             */
    float fsr_ns[3];           /* mean device ns per 4x4 block, fsr_blocks 4 / 2 / 8              */
} rfsr_tuning;

typedef struct {
    int height, width;     /* HR frame size (even, >= 16)                                        */
    int mask_type;         /* RFSR_MASK_FIXED / RFSR_MASK_DYNAMIC (informational)                 */
    int cc_mode;           /* RFSR_CC_*                                                          */
    int num_refs;          /* K, number of past frames for ME and projection, 0..3 (Sec. 4: 3)   */
    int template_size;     /* T, odd, 1..11 (default 9)                                          */
    int search_radius;     /* R, ME search window [-R, R]^2, 1..9 (default 8)                     */
    int check_radius;      /* Rc, RMC window [-Rc, Rc]^2, 1..9 (default = R)                     */
    int fsr_iterations;    /* FSR model iterations (default 100)                                 */
    float fsr_rho;         /* FSR spatial weighting decay (default 0.7)                          */
    float fsr_gamma;       /* FSR orthogonality deficiency compensation (default 0.5)            */
    float fsr_proj_weight; /* weight factor of projected pixels (default 1: same as measured)     */
    int fsr_overwrite_projected; /* 0: D-FSR (Sec. 3.2, default); 1: R-FSR overwrite          */
    int keep_f32;          /* 1: keep the FP32 FSR output of every frame for rfsr_get_frame      */
    float fsr_concealed_weight; /* delta >= 0 (default 0, Sec. 4: every block independent).  delta
                              > 0 is the original FSR: the pixels of blocks already reconstructed
                              in raster order that are neither measured nor projected join the
                              support with weight delta rho^d and their reconstruction as value;
                              blocks then run as wavefronts (block (i, j) after (i-1, j+4) and
                              (i, j-1)), one launch per wave, far slower.  On batched and serving
                              engines such a stream's FSR runs as its own wavefront launches right
                              after each batched step; rfsr_fsr_device then needs d_out_f32.     */
    int fsr_trace;         /* 1: record, for every 4x4 block of every frame, the basis pair the FSR
                              selected in each iteration (debug plane RFSR_DBG_FSR_SEL): the
                              selection is an argmax, so this makes the FP32 result checkable
                              against an FP64 replay of the same selections.  Costs
                              2 * iterations bytes per block of device memory.  0 (default): off */
    int me_predict_radius; /* 0 (default): every past frame gets the full ME search of Sec. 2.2.
                              Rp > 0: an opt-in variant that the paper does not describe and that
                              changes its results: frame t-k, k >= 2, is searched only within
                              radius Rp of the prediction k v_1(p) (v_1 = the vector to t-1,
                              clamped to [-R, R]^2 and into the frame), still inside [-R, R]^2,
                              same cost and tie order; Rp >= 2R equals the full search.  1..18;
                              needs template_size 9 and an unbatched engine (EINVAL otherwise) */
} rfsr_stream_config;

/* Fill a config with the defaults above (1280x720, NNC_FRMC, K=3, T=9, R=8). */
void rfsr_engine_config_default(rfsr_engine_config *cfg);
void rfsr_stream_config_default(rfsr_stream_config *cfg);

/* ---- engine ----------------------------------------------------------------------------- */
/* Create an engine on cfg->device.  *out is owned by the library until rfsr_engine_destroy.
 * Errors: EINVAL (NULL / bad field), EDEVICE (no such device, stream creation failed). */
int rfsr_engine_create(const rfsr_engine_config *cfg, rfsr_engine **out);
/* Waits for all work, destroys all streams of the engine and frees everything (EINVAL: NULL). */
int rfsr_engine_destroy(rfsr_engine *eng);
/* Batched engines: one frame step (Fig. 1) over every live stream that has a staged frame.
 * Each phase (ingest, ME, RME field, checks + projection, FSR) is one persistent launch over the
 * (stream, tile) pairs of all streams; the task-table copy and the launches are one CUDA graph
 * (captured at the first step of each template size, then replayed).  Host frames are read and
 * results written in mapped pinned memory by the kernels themselves.  Streams with more staged
 * frames get further steps in the same call.  Returns the number of frames launched (>= 0) or an
 * error (ESTATE: engine not batched). */
int rfsr_engine_step(rfsr_engine *eng);
/* Device time of the most recently launched batched step (waits for it) and its frame count.
 * Needs a batched engine created with profile = 1 (else ESTATE). */
int rfsr_engine_last_step_ms(rfsr_engine *eng, float *ms, int *frames);
/* Wait (bounded) until all launched work of the engine is done.  Errors: ETIMEDOUT, ESTATE
 * (a batched engine without a serving thread still has staged frames: call rfsr_engine_step). */
int rfsr_engine_sync(rfsr_engine *eng, int timeout_ms);
/* Batched engines: use this tile shape from the next step on (waits for the engine's launched
 * work, drops its captured graphs and ends autotuning).  Errors: EINVAL (shape not one of the
 * listed values), ESTATE (engine not batched). */
int rfsr_engine_set_shape(rfsr_engine *eng, const rfsr_batch_shape *shape);
/* Batched engines: the autotuner's state and measurements (ESTATE: engine not batched).  The
 * autotuner runs tuning step i with ME candidate i mod 3 (strips of 64 / 32 rows, box sums) and
 * FSR candidate i mod 3 (4 / 2 / 8 blocks), timing those two phases with CUDA events per unit of
 * work, and keeps per phase the fastest once each candidate has two measurements (at most 32
 * tuning steps). */
int rfsr_engine_get_tuning(rfsr_engine *eng, rfsr_tuning *out);

/* ---- streams (the four calls of the serving interface) ---------------------------------- */
/* Every call below that takes an engine accepts NULL for a process-wide default engine (default
 * configuration, created on first use on the calling thread's current device). */
/* Create a video stream.  The stream owns its device state: K+1 ring slots of reconstruction,
 * sample plane and mask, the motion fields, decisions, projection sums and FSR output.  If that
 * state does not fit the engine's memory budget now, the stream is queued: *out is set and the
 * call returns EAGAIN; the stream becomes live (rfsr_stream_get_info: live = 1) when enough
 * streams have been destroyed, in arrival order; until then pushes return EAGAIN.
 * Errors: EINVAL (sizes / parameters), ENOMEM (the stream alone exceeds the budget, or device
 * memory ran out), EDEVICE.  *out is owned by the library until rfsr_destroy. */
int rfsr_create_stream(rfsr_engine *eng, const rfsr_stream_config *cfg, rfsr_stream **out);

/* Push frame t: samples = f_sub (H x W, unmeasured bytes ignored), mask = b (H x W, 0/1, one 1
 * per 2x2 block), both HOST memory owned by the caller and copied before return, so the caller
 * may reuse them at once.  The frame step runs asynchronously on the GPU (batched engines: at the
 * next rfsr_engine_step, or at once in a serving engine).
 * Errors: EINVAL, EMASK (checked on the host before anything is enqueued; the stream state is
 * unchanged), EBUSY (max_inflight frames not yet collected), EAGAIN (stream still queued),
 * EDEVICE. */
int rfsr_push_frame(rfsr_stream *s, const uint8_t *samples, const uint8_t *mask);

/* As rfsr_push_frame, but samples and mask are DEVICE buffers (2-byte aligned, else EINVAL) that
 * must stay unchanged until the frame has been collected (rfsr_get_frame / rfsr_get_frame_device
 * returned it).  producer_stream is the cudaStream_t on which the caller wrote them: the engine's
 * work waits for what was enqueued there up to this call (an event, no host wait); NULL means
 * the buffers are already complete.  The mask is validated on the GPU; a bad mask is reported as
 * EMASK by the call that collects the frame, and the frame then leaves the stream's history
 * unchanged. */
int rfsr_push_frame_device(rfsr_stream *s, const uint8_t *samples, const uint8_t *mask,
                           void *producer_stream);

/* Collect the oldest uncollected frame (FIFO): out_u8 = 8-bit reconstruction (H x W host),
 * out_f32 = FSR output on the [0, 1] scale before quantisation (H x W host, may be NULL; needs
 * keep_f32).  Waits at most timeout_ms (< 0: no limit) and never hangs beyond that.
 * Errors: ESTATE (nothing pushed), ETIMEDOUT, EMASK (frame had a bad device mask), EINVAL. */
int rfsr_get_frame(rfsr_stream *s, uint8_t *out_u8, float *out_f32, int timeout_ms);

/* As rfsr_get_frame, into DEVICE buffers (either may be NULL). */
int rfsr_get_frame_device(rfsr_stream *s, uint8_t *d_out_u8, float *d_out_f32, int timeout_ms);

/* Destroy a stream.  Waits for its frames in flight, then frees its device and host state.
 * A queued stream leaves the admission queue.  Errors: EINVAL (NULL). */
int rfsr_destroy(rfsr_stream *s);

/* ---- state, history injection and debug planes (parity tests, checkpointing) ------------ */
typedef struct {
    int height, width;
    int live;              /* 1 when admitted (0 while queued by memory admission)               */
    long long frames_pushed, frames_collected;
    int history_frames;    /* past frames available to the next frame (0..K)                      */
    size_t device_bytes;   /* device memory held by this stream                                   */
} rfsr_stream_info;
int rfsr_stream_get_info(rfsr_stream *s, rfsr_stream_info *info);   /* EINVAL: NULL argument */
/* Admission state of s: 1 live, 0 queued for memory (rfsr_create_stream returned EAGAIN),
 * negative on error (EINVAL: NULL stream). */
int rfsr_stream_state(rfsr_stream *s);

/* Replace the history seen by the next pushed frame: for k = 1..nrefs, rec[k-1], smp[k-1] and
 * msk[k-1] are the reconstruction, sample plane and 0/1 mask of frame t-k (HOST buffers, H x W,
 * copied before return).  nrefs <= K.  Waits for the stream's frames in flight first. */
int rfsr_set_history(rfsr_stream *s, int nrefs, const uint8_t *const *rec,
                     const uint8_t *const *smp, const uint8_t *const *msk);

/* Debug planes of the most recently completed frame (waits for it), copied to HOST memory dst:
 *   RFSR_DBG_MV        k in 1..K_eff: raw ME field, H*W*2 int8 (vertical, horizontal)
 *   RFSR_DBG_FMV       k: vector used by checks and projection (NNC median when NNC is on)
 *   RFSR_DBG_DECISION  k: H*W uint8 RFSR_DEC_* labels
 *   RFSR_DBG_PSUM      projection sums, H*W uint16;  RFSR_DBG_PCNT counts, H*W uint8
 *   RFSR_DBG_FSR       FSR output, H*W float;        RFSR_DBG_REC reconstruction, H*W uint8
 *   RFSR_DBG_RMV       k: reverse ME field at every past-frame pixel (RME mode only)
 *   RFSR_DBG_FSR_SEL   FSR selections (streams with fsr_trace = 1): nblocks * fsr_iterations
 *                      uint16, block-major over the row-major 4x4 blocks (ceil(H/4) x ceil(W/4));
 *                      entry i of a block is the canonical linear index k*32 + l of the basis
 *                      pair selected in iteration i (Sec. 2.1: one pair per iteration), or
 *                      RFSR_FSR_SEL_NONE where the block ran no iteration i (W(0) = 0 or the
 *                      residual was exhausted)
 * Errors: ESTATE (no frame done yet, k > K_eff of that frame, plane not recorded), EINVAL. */
enum { RFSR_DBG_MV = 0, RFSR_DBG_FMV = 1, RFSR_DBG_DECISION = 2, RFSR_DBG_PSUM = 3,
       RFSR_DBG_PCNT = 4, RFSR_DBG_FSR = 5, RFSR_DBG_REC = 6, RFSR_DBG_RMV = 7,
       RFSR_DBG_FSR_SEL = 8 };
#define RFSR_FSR_SEL_NONE 0xffffu
int rfsr_debug_get(rfsr_stream *s, int what, int k, void *dst);

/* ---- stand-alone FSR (Sec. 2.1, 3.2) on device buffers ---------------------------------- */
/* Reconstruct every 4x4 block of an H x W frame from its 32x32 support.  d_smp: sample plane
 * (H*W uint8), d_msk: 0/1 mask (H*W uint8), d_psum / d_pcnt: projection sums and counts (H*W
 * uint16 / uint8, both NULL for single-frame FSR; d_psum 2-byte aligned).  Outputs: d_out_f32
 * (H*W float, [0,1] scale, 4-byte aligned, may be NULL) and d_out_u8 (H*W uint8, may be NULL).
 * cfg supplies the fsr_* fields and height / width.  Runs on cuda_stream (cudaStream_t,
 * NULL = legacy default stream) and returns
 * without waiting.  Errors: EINVAL, EDEVICE. */
int rfsr_fsr_device(const rfsr_stream_config *cfg, const uint8_t *d_smp, const uint8_t *d_msk,
                    const uint16_t *d_psum, const uint8_t *d_pcnt, float *d_out_f32,
                    uint8_t *d_out_u8, void *cuda_stream);

/* As rfsr_fsr_device, and also records the selected basis pair of every iteration of every block
 * in d_sel (device, nblocks * cfg->fsr_iterations uint16, 2-byte aligned; layout and
 * RFSR_FSR_SEL_NONE as for RFSR_DBG_FSR_SEL).  The model update of Sec. 2.1 depends on the
 * selections only, so an FP64 evaluation that follows the same selections reproduces the FP32
 * output to rounding; this is how FP32 results at near-tied selections are checked.  Same errors
 * as rfsr_fsr_device (EINVAL also for a NULL or misaligned d_sel). */
int rfsr_fsr_device_trace(const rfsr_stream_config *cfg, const uint8_t *d_smp,
                          const uint8_t *d_msk, const uint16_t *d_psum, const uint8_t *d_pcnt,
                          float *d_out_f32, uint8_t *d_out_u8, uint16_t *d_sel,
                          void *cuda_stream);

/* ---- stream state: checkpoint / resume and migration between engines -------------------- */
/* (No counterpart in the paper: serving infrastructure.)  The recursion state of a stream is
 * its configuration and the reconstructed frame, sample plane and mask of its last K frames
 * (Sec. 2.2: the past frames that ME and projection read).  rfsr_stream_export writes it to a
 * caller-owned host buffer; rfsr_stream_import creates a stream from it on any engine (another
 * GPU included), whose next frame then gives exactly the result the original stream would have.
 * Buffer layout: rfsr_state_header, then for k = 1..hist the planes of frame t-k
 * (reconstruction, samples, 0/1 mask; H x W bytes each, row-major). */
typedef struct {
    uint32_t magic;              /* RFSR_STATE_MAGIC                                               */
    uint32_t version;            /* RFSR_STATE_VERSION                                             */
    uint64_t bytes;              /* size of the whole buffer                                       */
    rfsr_stream_config config;   /* the stream's configuration                                     */
    int32_t hist;                /* past frames stored (0..num_refs)                               */
    int32_t reserved;
    int64_t frames;              /* frames the exported stream had processed                       */
} rfsr_state_header;
#define RFSR_STATE_MAGIC 0x54534652u   /* "RFST" */
#define RFSR_STATE_VERSION 4u

/* Export s into buf (cap bytes); *bytes receives the size needed (buf == NULL: size query).
 * Taken between frames: every pushed frame must have been collected.
 * Errors: EINVAL (NULL bytes, cap too small), EAGAIN (stream still queued), ESTATE (frames not
 * yet collected, or the stream had a bad mask), EDEVICE. */
int rfsr_stream_export(rfsr_stream *s, void *buf, size_t cap, size_t *bytes);
/* Create a stream on eng from an exported state.  *out is owned by the library until
 * rfsr_destroy.  Errors: EINVAL (not a state buffer of this version, inconsistent size or
 * configuration), ENOMEM, EAGAIN (the engine's memory budget is full now: nothing is created,
 * retry later), EMASK, EDEVICE. */
int rfsr_stream_import(rfsr_engine *eng, const void *buf, size_t bytes, rfsr_stream **out);

/* Engine occupancy for placement decisions (rfsr_engine_get_info). */
typedef struct {
    int device;
    size_t memory_budget;        /* bytes of device memory streams may use                         */
    size_t memory_used;          /* bytes held by live streams                                     */
    int streams_live;
    int streams_queued;
} rfsr_engine_info;
int rfsr_engine_get_info(rfsr_engine *eng, rfsr_engine_info *info);   /* EINVAL: NULL argument */

/* Device time of the phases of the most recently pushed frame of s (waits for it), measured with
 * CUDA events on the engine's stream around each kernel: ms[0] ingest, ms[1] motion estimation,
 * ms[2] consistency checks (with the RME reverse field) + projection, ms[3] FSR + 8-bit
 * reconstruction.
 * Needs an engine created with profile = 1 (else ESTATE). */
int rfsr_stream_phase_ms(rfsr_stream *s, float ms[4]);

/* ---- one frame of ME + checks + projection without allocating device memory ------------- */
/* The paper has no counterpart to this call; it exists for callers that cannot allocate device
 * memory while they run -- a real-time loop that must keep allocator locks and driver
 * allocations out of its latency, a plugin inside an application that owns all of the GPU's
 * memory and hands out only buffers it created, or code that may not allocate after start-up.
 * It computes what one frame step computes up to the projection (ingest, motion estimation
 * against nrefs past frames, the checks of cfg->cc_mode, projection sums and counts), writing
 * only the caller's outputs, and calls no cudaMalloc / cudaFree or any allocating routine.
 * Every intermediate plane lives in one fixed array of 8 MiB in the library's static device
 * memory, which each GPU that loads the library holds until the process exits.  A frame fits if
 *     256 + 2*A(H*W) + nrefs*(2*A(2*H*W) + A(H*W)) [+ nrefs*A(2*H*W) in RME mode] <= 8 MiB,
 * A(n) = n rounded up to a multiple of 256 (e.g. 640x480 with three past frames in any mode);
 * larger frames are rejected with EINVAL and a message giving the bytes needed.
 *   cfg: height, width, cc_mode, template_size, search_radius, check_radius (FSR fields unused)
 *   d_smp, d_msk: current sample plane and 0/1 mask (H*W uint8, device, 2-byte aligned)
 *   d_ref_rec[k], d_ref_smp[k], d_ref_msk[k] (k < nrefs <= 3): HOST arrays of DEVICE pointers
 *       to the reconstruction, sample plane and 0/1 mask of frame t-1-k (H*W uint8 each)
 *   d_psum, d_pcnt: outputs, projection sums (H*W uint16, 2-byte aligned) and counts (H*W uint8)
 *   d_dec: optional output, nrefs*H*W RFSR_DEC_* labels (k-major); d_status: optional output,
 *       one int (4-byte aligned) set to 0 when d_msk is a quarter-sampling mask and to 1 when it
 *       is not (the other outputs are then left unwritten)
 *   cuda_stream: cudaStream_t to run on (NULL = legacy default stream); returns without waiting.
 * It runs on the calling thread's current device.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) for that device; make that first call before
 * any stream capture.  All calls share the one array, which keeps the last call's contents, so
 * calls whose work overlaps on the GPU (other streams, other threads) race: serialise them.
 * Errors: EINVAL (NULL / misaligned / out-of-range arguments, frame too large), EDEVICE. */
int rfsr_me_cc_project_noalloc(const rfsr_stream_config *cfg, const uint8_t *d_smp,
                               const uint8_t *d_msk, int nrefs, const uint8_t *const *d_ref_rec,
                               const uint8_t *const *d_ref_smp, const uint8_t *const *d_ref_msk,
                               uint16_t *d_psum, uint8_t *d_pcnt, uint8_t *d_dec, int *d_status,
                               void *cuda_stream);

/* Throughput probe for roofline denominators (not part of the method): runs a chain of one
 * instruction kind on every SM of `device` and returns instructions per second and per clock per
 * SM.  kind: 0 3-input add, 1 3-input logic, 2 byte permute, 3 byte |a-b| (__vabsdiffu4),
 * 4 byte SAD (__vsadu4) + add, 5 16-bit x2 3-way max, 6 16-bit x2 3-way min, 7 integer multiply-add,
 * 8 |a-b|+c (__sad), 9 32-bit min, 10 xor, 11 FP32 fused multiply-add, 12 3-input adds and
 * integer multiply-adds interleaved (one each per pair of chains), 13 byte SAD with accumulate
 * (one vabsdiff4.add), 14 signed 16-bit x2 minimum (min.s16x2), 15 sum of the two signed 16-bit
 * |a-b| with accumulate (vabsdiff2.add), 16 signed 16-bit x2 3-way max, 17 32-bit 3-way max.
 * Synchronous; allocates
 * and frees its own small buffers.  Errors: EINVAL, EDEVICE. */
int rfsr_alu_peak(int device, int kind, int iters, double *ops_per_sec, double *ops_per_clk_sm);

/* Kernel launches made by this process so far (all engines), for launch accounting. */
long long rfsr_kernel_launches(void);

/* Inspection (no counterpart in the paper): the order in which the CTAs of the fused ME + checks
 * launch (engine option fuse_me_cc) claim the tiles of a height x width frame with num_refs past
 * frames on a grid of `grid` CTAs.  Item: bit 31 set for a check tile (32 x 32 pixels at tile
 * column bits 0..9, tile row bits 10..21), clear for an ME tile (64-row band bits 10..21, 120-column
 * tile bits 0..9, past frame bits 22..23).  A check tile reads the motion fields of rows
 * 32 row - 2 .. 32 row + 33; the launch relies on every ME tile of those rows' bands coming earlier
 * in the order.  Pure host code.  Writes up to `capacity` items (items may be NULL) and returns
 * the count, or EINVAL for bad sizes. */
int rfsr_fused_schedule(int height, int width, int num_refs, int grid, uint32_t *items,
                        int capacity);

/* Message of the last failed call on this thread ("" if none). */
const char *rfsr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RFSR_H */
