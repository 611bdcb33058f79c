// rfsr_api.cpp -- the C ABI declared in include/rfsr.h: engines, streams with their device-
// resident state, the asynchronous frame step, batching and serving.
//
// A stream keeps everything the recursion needs on the device (Sec. 2.2 / Fig. 1): a ring of
// K+1 slots holding the reconstruction, sample plane and mask of the current and the K previous
// frames, the per-reference motion fields, decisions, projection sums and the FSR output.  A
// frame step is one sequence of kernels on the engine's CUDA stream:
//     ingest -> ME (all K references in one launch) -> [RME reverse field] -> checks + projection
//     -> FSR + 8-bit reconstruction
//
// Unbatched engines launch a stream's step when its frame is pushed, preceded (host push) by one
// pinned host->device copy of the frame and followed by one device->host copy of the result.
//
// Batched engines stage pushed frames and run one step over every stream that has one: a task
// table (one FrameTask per stream) is copied to the device and each phase is one persistent
// launch over the (stream, tile) pairs of all tasks; the copy and the launches are captured once
// in a CUDA graph per template size and replayed.  Host frames are read by the ingest kernel and
// results written by the FSR kernel directly in mapped pinned memory, so a batched step issues
// no per-stream copies.  Streams whose state does not fit the engine's memory budget are queued
// (EAGAIN) and admitted when memory frees.  With serve = 1 an engine thread launches a batched
// step whenever frames are staged (continuous batching: frames that arrive while a step runs go
// into the next one).
#include "rfsr.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rfsr_internal.h"

using namespace rfsr;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return RFSR_EDEVICE;
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

// host-side quarter-sampling check (Sec. 1): values 0/1 and exactly one 1 per 2x2 block.  Eight
// columns of two rows at a time: every byte <= 1, and each 2x2 block sums to one.
bool mask_ok(const uint8_t *m, int H, int W)
{
    constexpr uint64_t kHigh = 0xfefefefefefefefeull, kLow = 0x00ff00ff00ff00ffull;
    constexpr uint64_t kOne = 0x0001000100010001ull;
    for (int y = 0; y < H; y += 2) {
        const uint8_t *r0 = m + (size_t)y * W, *r1 = r0 + W;
        int x = 0;
        for (; x + 8 <= W; x += 8) {
            uint64_t a, b;
            std::memcpy(&a, r0 + x, 8);
            std::memcpy(&b, r1 + x, 8);
            if ((a | b) & kHigh) return false;                    // a byte other than 0 / 1
            const uint64_t s = a + b;                             // column sums 0..2 per byte
            if (((s + (s >> 8)) & kLow) != kOne) return false;    // pairs of columns: one each
        }
        for (; x < W; x += 2) {
            const unsigned a = r0[x], b = r0[x + 1], c = r1[x], d = r1[x + 1];
            if (((a | b | c | d) & ~1u) || a + b + c + d != 1) return false;
        }
    }
    return true;
}

// FSR tables (Sec. 2.1 model): rho^d over the support, frequency weights, DFT twiddles.
void fill_fsr_tables(FsrTables &tb, double rho)
{
    const int N = kFsrN;
    const double c = (N - 1) / 2.0;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n)
            tb.wsp[m * N + n] = (float)std::pow(rho, std::sqrt((m - c) * (m - c) + (n - c) * (n - c)));
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < kFsrHalf; ++l) {
            const double kn = std::min(k, N - k) / (N / 2.0), ln = std::min(l, N - l) / (N / 2.0);
            const double v = 1.0 - std::sqrt(2.0) / 2.0 * std::sqrt(kn * kn + ln * ln);
            tb.wf[k * kFsrHalf + l] = (float)(v * v);
        }
    for (int j = 0; j < N; ++j) {
        tb.cs[j] = (float)std::cos(2.0 * M_PI * j / N);
        tb.sn[j] = (float)std::sin(2.0 * M_PI * j / N);
    }
}

using Clock = std::chrono::steady_clock;

// bounded wait on an event: polls (never blocks inside the CUDA runtime) and gives up after
// timeout_ms
int wait_event(cudaEvent_t ev, int timeout_ms, Clock::time_point t0 = Clock::now())
{
    int spins = 0;
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return RFSR_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(RFSR_ETIMEDOUT, "frame not ready within timeout");
        }
        if (++spins < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

int rfsr::set_error(int code, const std::string &msg) { return fail(code, msg); }

bool rfsr::shape_valid(const BatchShape &s)
{
    return (s.me_warps == 4 || s.me_warps == 8) && (s.me_box == 0 || s.me_box == 1) &&
           (s.fsr_blocks == 2 || s.fsr_blocks == 4 || s.fsr_blocks == 8);
}

struct Slot {
    uint8_t *h_in = nullptr;    // pinned, mapped: samples | mask
    uint8_t *h_in_dev = nullptr;
    uint8_t *d_in = nullptr;    // device samples | mask (unbatched host pushes)
    uint8_t *h_out = nullptr;   // pinned, mapped: reconstruction
    uint8_t *h_out_dev = nullptr;
    float *h_out32 = nullptr;   // pinned FSR output (keep_f32)
    uint8_t *d_out = nullptr;   // device reconstruction
    float *d_out32 = nullptr;   // device FSR output (keep_f32)
    int *d_status = nullptr;
    int *h_status = nullptr;    // pinned, mapped
    int *h_status_dev = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t ready = nullptr;  // device pushes: recorded on the producer's stream
    bool wait_ready = false;      // the engine's stream must wait for `ready` before this frame
    cudaEvent_t phase[5] = {};  // profile: before ingest, after ingest / ME / checks / FSR
    bool host_push = false;
    const uint8_t *in_smp = nullptr;   // staged input of a batched engine (device-visible)
    const uint8_t *in_msk = nullptr;
};

struct BatchSet {                      // one of two alternating batch buffers
    BatchDesc *h = nullptr;            // pinned staging
    BatchDesc *d = nullptr;            // device copy the kernels read
    cudaEvent_t done = nullptr;        // recorded after the batch's last kernel
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // timing events around the batch (profile)
    cudaEvent_t ph[4] = {};            // tuning: before / after ME, before / after FSR
    std::map<int, cudaGraphExec_t> graphs;    // key 2*T + rme
    std::map<int, int> graph_kernels;
    bool used = false;
    bool tune_pending = false;         // a tuning measurement waits in ph[]
    int tune_me = -1, tune_fsr = -1;   // candidates it measured (-1: phase not measured)
    double me_units = 0, fsr_units = 0;
};

// Online autotuner of the batched tile shapes.  Every shape gives bit-identical results, so the
// first batched steps of an engine serve as the measurements: tuning step i runs ME (T = 9) with
// candidate i mod 2 and FSR with candidate i mod 3, directly launched with events around the two
// phases.  Once every candidate has kSamples measurements the engine keeps, per phase, the one
// with the least device time per unit of work (ME: pixel x reference, FSR: 4x4 block); from then
// on its steps are captured and replayed as CUDA graphs.
struct Tuner {
    static constexpr int kMe = 3, kFsr = 3, kSamples = 2, kMaxSteps = 32;
    static constexpr int me_cand[kMe] = {8, 4, 0};       // warp strips per ME tile (64 / 32 rows);
                                                         // 0: the sliding-window box-sum kernel
    static constexpr int fsr_cand[kFsr] = {4, 2, 8};     // FSR blocks per CTA
    bool active = false;
    int steps = 0;                                       // tuning steps launched
    int measured = 0;                                    // tuning steps harvested
    double me_ns[kMe] = {}, fsr_ns[kFsr] = {};           // sums of ns per unit
    int me_n[kMe] = {}, fsr_n[kFsr] = {};
};

struct rfsr_engine {
    rfsr_engine_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::vector<rfsr_stream *> streams;        // live and queued
    std::deque<rfsr_stream *> queued;          // waiting for memory, in arrival order
    BatchSet sets[2];
    int next_set = 0;
    bool graphs_ok = true;
    BatchShape shape;                          // tile shapes of the batched launches
    Tuner tune;
    long long staged = 0;                      // frames pushed but not launched (batched)
    long long batches = 0;
    int last_batch_set = -1, last_batch_frames = 0;
    std::thread server;
    std::condition_variable cv;
    bool stop = false;
};

struct rfsr_stream {
    rfsr_engine *eng = nullptr;
    rfsr_stream_config cfg{};
    int H = 0, W = 0, K = 0;
    size_t bytes = 0, need = 0;
    bool live = false;
    std::vector<void *> dev_allocs;
    std::vector<void *> host_allocs;
    uint8_t *ring_rec[kMaxRefs + 1] = {}, *ring_smp[kMaxRefs + 1] = {}, *ring_msk[kMaxRefs + 1] = {};
    int8_t *mv[kMaxRefs] = {}, *fmv[kMaxRefs] = {}, *rmv[kMaxRefs] = {};
    uint8_t *dec[kMaxRefs] = {};
    uint16_t *psum = nullptr;
    uint8_t *pcnt = nullptr;
    float *fsr = nullptr;
    uint16_t *fsr_sel = nullptr;   // selection trace (fsr_trace streams)
    // fused ME + checks launch: claim orders for 1..K past frames, counters
    uint32_t *mecc_items = nullptr;
    int mecc_off[kMaxRefs + 1] = {}, mecc_n[kMaxRefs + 1] = {};
    int *mecc_ctr = nullptr;
    int mecc_nb = 0;
    float *tables = nullptr;
    int *d_zero = nullptr;
    std::vector<Slot> slots;
    long long pushed = 0, launched = 0, collected = 0;
    int hist = 0;          // history frames available to the next frame
    int ring_head = 0;     // ring index of the next frame
    int last_slot = -1, last_ring = -1, last_K = 0;
    bool poisoned = false;

    int dev_alloc(void **p, size_t n)
    {
        const rfsr_engine_config &c = eng->cfg;
        if (c.dev_alloc) {
            *p = c.dev_alloc(n, c.alloc_ctx);
            if (!*p) return fail(RFSR_ENOMEM, "dev_alloc callback returned NULL");
        } else {
            cudaError_t e = cudaMalloc(p, n);
            if (e != cudaSuccess)
                return fail(RFSR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        dev_allocs.push_back(*p);
        bytes += n;
        return RFSR_OK;
    }
    int host_alloc(void **p, size_t n)
    {
        cudaError_t e = cudaHostAlloc(p, n, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return fail(RFSR_ENOMEM, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
        host_allocs.push_back(*p);
        return RFSR_OK;
    }
    void release()
    {
        for (auto &s : slots) {
            if (s.done) cudaEventDestroy(s.done);
            if (s.ready) cudaEventDestroy(s.ready);
            for (auto &ev : s.phase)
                if (ev) cudaEventDestroy(ev);
        }
        for (void *p : dev_allocs) {
            if (eng->cfg.dev_free) eng->cfg.dev_free(p, eng->cfg.alloc_ctx);
            else cudaFree(p);
        }
        for (void *p : host_allocs) cudaFreeHost(p);
        dev_allocs.clear();
        host_allocs.clear();
        slots.clear();
        bytes = 0;
    }
};

namespace {

bool batched(const rfsr_engine *e) { return e->cfg.batched || e->cfg.serve; }

// bytes of the FSR selection trace of one frame (0 unless the stream records it)
size_t trace_bytes(const rfsr_stream_config *c)
{
    if (!c->fsr_trace) return 0;
    const size_t nb = (size_t)((c->height + kFsrB - 1) / kFsrB) * ((c->width + kFsrB - 1) / kFsrB);
    return std::max<size_t>(2, 2 * nb * (size_t)c->fsr_iterations);
}

// frame steps of this stream run ME and the checks as one fused launch (engines that ask for it;
// unbatched, T = 9, full ME search, no RME)
bool fused_me_cc(const rfsr_engine_config &e, const rfsr_stream_config *c)
{
    return !e.batched && !e.serve && e.fuse_me_cc && c->template_size == 9 &&
           c->cc_mode != RFSR_CC_RME && c->me_predict_radius == 0 && c->num_refs > 0;
}

// bytes of the fused launch's claim orders (1..K past frames) and counters
size_t mecc_bytes(const rfsr_stream_config *c)
{
    size_t n = 0;
    for (int k = 1; k <= c->num_refs; ++k) n += (size_t)mecc_schedule(c->height, c->width, k, 1, nullptr);
    return 4 * n + 4 * (size_t)(mecc_bands(c->height) + 3);
}

// device bytes a stream will hold (admission against the engine budget)
size_t stream_need(const rfsr_stream_config *c, int M, bool fused)
{
    const size_t HW = (size_t)c->height * c->width;
    const int K = c->num_refs;
    const bool rme = c->cc_mode == RFSR_CC_RME;
    return (size_t)(K + 1) * 3 * HW + (size_t)K * (2 * HW * (rme ? 3 : 2) + HW) + 3 * HW + 4 * HW +
           sizeof(FsrTables) + 64 + (size_t)M * (3 * HW + (c->keep_f32 ? 4 * HW : 0) + 4) +
           trace_bytes(c) + (fused ? mecc_bytes(c) : 0);
}

// allocate a stream's device and pinned state (engine lock held)
int admit(rfsr_stream *s)
{
    rfsr_engine *e = s->eng;
    const size_t HW = (size_t)s->H * s->W;
    const int M = e->cfg.max_inflight;
    const bool rme = s->cfg.cc_mode == RFSR_CC_RME;
    auto bail = [&](int code) {
        s->release();
        return code;
    };
#define AL(ptr, n)                                                 \
    do {                                                           \
        int r_ = s->dev_alloc((void **)&(ptr), (n));               \
        if (r_) return bail(r_);                                   \
    } while (0)
    for (int r = 0; r <= s->K; ++r) {
        AL(s->ring_rec[r], HW);
        AL(s->ring_smp[r], HW);
        AL(s->ring_msk[r], HW);
    }
    for (int k = 0; k < s->K; ++k) {
        AL(s->mv[k], 2 * HW);
        AL(s->fmv[k], 2 * HW);
        AL(s->dec[k], HW);
        if (rme) AL(s->rmv[k], 2 * HW);
    }
    AL(s->psum, 2 * HW);
    AL(s->pcnt, HW);
    AL(s->fsr, 4 * HW);
    if (s->cfg.fsr_trace) AL(s->fsr_sel, trace_bytes(&s->cfg));
    AL(s->tables, sizeof(FsrTables));
    AL(s->d_zero, 64);
    cudaError_t er = cudaMemset(s->d_zero, 0, 64);
    if (er != cudaSuccess) return bail(cuda_fail(er, "cudaMemset"));
    if (fused_me_cc(e->cfg, &s->cfg)) {                // claim orders of the fused ME + checks launch
        const int grid = mecc_grid();
        if (grid <= 0) return bail(fail(RFSR_EDEVICE, "fused ME + checks launch: no resident grid"));
        std::vector<uint32_t> items;
        for (int k = 1; k <= s->K; ++k) {
            const int n = mecc_schedule(s->H, s->W, k, grid, nullptr);
            s->mecc_off[k] = (int)items.size();
            s->mecc_n[k] = n;
            items.resize(items.size() + n);
            mecc_schedule(s->H, s->W, k, grid, items.data() + s->mecc_off[k]);
        }
        s->mecc_nb = mecc_bands(s->H);
        AL(s->mecc_items, 4 * items.size());
        AL(s->mecc_ctr, 4 * (size_t)(s->mecc_nb + 3));
        er = cudaMemcpy(s->mecc_items, items.data(), 4 * items.size(), cudaMemcpyHostToDevice);
        if (er != cudaSuccess) return bail(cuda_fail(er, "cudaMemcpy claim order"));
    }
    {
        FsrTables tb;
        fill_fsr_tables(tb, s->cfg.fsr_rho);
        er = cudaMemcpy(s->tables, &tb, sizeof(tb), cudaMemcpyHostToDevice);
        if (er != cudaSuccess) return bail(cuda_fail(er, "cudaMemcpy tables"));
    }
    s->slots.assign(M, Slot());
    for (int i = 0; i < M; ++i) {
        Slot &sl = s->slots[i];
        AL(sl.d_in, 2 * HW);
        AL(sl.d_out, HW);
        AL(sl.d_status, 4);
        if (s->cfg.keep_f32) AL(sl.d_out32, 4 * HW);
        int r_ = s->host_alloc((void **)&sl.h_in, 2 * HW);
        if (!r_) r_ = s->host_alloc((void **)&sl.h_out, HW);
        if (!r_) r_ = s->host_alloc((void **)&sl.h_status, 64);
        if (!r_ && s->cfg.keep_f32) r_ = s->host_alloc((void **)&sl.h_out32, 4 * HW);
        if (r_) return bail(r_);
        er = cudaHostGetDevicePointer((void **)&sl.h_in_dev, sl.h_in, 0);
        if (er == cudaSuccess) er = cudaHostGetDevicePointer((void **)&sl.h_out_dev, sl.h_out, 0);
        if (er == cudaSuccess) er = cudaHostGetDevicePointer((void **)&sl.h_status_dev, sl.h_status, 0);
        if (er != cudaSuccess) return bail(cuda_fail(er, "cudaHostGetDevicePointer"));
        *sl.h_status = 0;
        er = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (er == cudaSuccess) er = cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming);
        if (er != cudaSuccess) return bail(cuda_fail(er, "cudaEventCreate"));
        if (e->cfg.profile)
            for (auto &ev : sl.phase) {
                er = cudaEventCreate(&ev);
                if (er != cudaSuccess) return bail(cuda_fail(er, "cudaEventCreate"));
            }
    }
#undef AL
    s->live = true;
    return RFSR_OK;
}

// admit queued streams in arrival order while they fit (engine lock held)
void admit_queued(rfsr_engine *e)
{
    while (!e->queued.empty()) {
        rfsr_stream *s = e->queued.front();
        if (e->used + s->need > e->budget) break;
        e->used += s->need;
        if (admit(s) != RFSR_OK) {          // device memory is short after all: keep it queued
            e->used -= s->need;
            break;
        }
        e->queued.pop_front();
    }
}

// the FrameTask of a stream's next frame; advances the ring (engine lock held)
void prepare_frame(rfsr_stream *s, int slot_idx, const uint8_t *in_smp, const uint8_t *in_msk,
                   FrameTask &t)
{
    Slot &sl = s->slots[slot_idx];
    std::memset(&t, 0, sizeof(t));
    const int R1 = s->K + 1;
    const int r = s->ring_head;
    t.H = s->H;
    t.W = s->W;
    t.K = s->hist;
    t.T = s->cfg.template_size;
    t.R = s->cfg.search_radius;
    t.Rc = s->cfg.check_radius;
    t.me_pred = s->cfg.me_predict_radius;
    t.cc_mode = s->cfg.cc_mode;
    t.fsr_iters = s->cfg.fsr_iterations;
    t.fsr_gamma = s->cfg.fsr_gamma;
    t.fsr_concealed = s->cfg.fsr_concealed_weight;
    t.fsr_proj_weight = s->cfg.fsr_proj_weight;
    t.fsr_overwrite_projected = s->cfg.fsr_overwrite_projected;
    t.fsr_tables = s->tables;
    t.in_smp = in_smp;
    t.in_msk = in_msk;
    t.cur_smp = s->ring_smp[r];
    t.cur_msk = s->ring_msk[r];
    t.cur_rec = s->ring_rec[r];
    for (int k = 1; k <= t.K; ++k) {
        const int rr = ((r - k) % R1 + R1) % R1;
        t.ref_rec[k - 1] = s->ring_rec[rr];
        t.ref_smp[k - 1] = s->ring_smp[rr];
        t.ref_msk[k - 1] = s->ring_msk[rr];
        t.mv[k - 1] = s->mv[k - 1];
        t.fmv[k - 1] = s->fmv[k - 1];
        t.dec[k - 1] = s->dec[k - 1];
        t.rmv[k - 1] = s->rmv[k - 1];
    }
    t.psum = s->psum;
    t.pcnt = s->pcnt;
    t.fsr_out = sl.d_out32 ? sl.d_out32 : s->fsr;
    t.out_u8 = sl.d_out;
    t.status = sl.d_status;
    t.prev_status = s->last_slot >= 0 ? s->slots[s->last_slot].d_status : s->d_zero;
    t.status_out = nullptr;
    t.fsr_sel = s->fsr_sel;
    s->last_K = t.K;
    s->last_ring = s->ring_head;
    s->last_slot = slot_idx;
    s->ring_head = (s->ring_head + 1) % (s->K + 1);
    s->hist = std::min(s->hist + 1, s->K);
}

// unbatched: the whole frame step of one stream on the engine stream
int enqueue_step(rfsr_stream *s, int slot_idx, const uint8_t *in_smp, const uint8_t *in_msk)
{
    rfsr_engine *e = s->eng;
    Slot &sl = s->slots[slot_idx];
    FrameTask t;
    prepare_frame(s, slot_idx, in_smp, in_msk, t);
    const bool prof = e->cfg.profile != 0;
    const bool fused = s->mecc_items != nullptr && t.K > 0;
    CK(cudaMemsetAsync(sl.d_status, 0, sizeof(int), e->stream));
    if (fused) CK(cudaMemsetAsync(s->mecc_ctr, 0, sizeof(int) * (size_t)(s->mecc_nb + 3), e->stream));
    if (prof) CK(cudaEventRecord(sl.phase[0], e->stream));
    CK(launch_ingest(t, e->stream));
    if (prof) CK(cudaEventRecord(sl.phase[1], e->stream));
    if (fused) {                                     // ME, checks and projection in one launch
        MeccPlan m;
        m.items = s->mecc_items + s->mecc_off[t.K];
        m.nitems = s->mecc_n[t.K];
        m.ctr = s->mecc_ctr;
        m.nbands = s->mecc_nb;
        m.need = mecc_need(t.W, t.K);
        m.limit = e->cfg.wait_test ? 4096 : (1 << 21);   // polls of about 0.5 us: 2 ms / 1 s
        m.bias = e->cfg.wait_test ? 1 : 0;
        m.status = t.status;
        FrameTask tf = t;                            // the tiles see a status word that stays 0
        tf.status = s->mecc_ctr + s->mecc_nb + 2;
        CK(launch_me_cc(tf, m, e->stream));
        if (prof) CK(cudaEventRecord(sl.phase[2], e->stream));
    } else {
        CK(launch_me(t, e->stream));
        if (prof) CK(cudaEventRecord(sl.phase[2], e->stream));
        // the reverse field of RME belongs to the consistency check (Sec. 2.2), so it is timed there
        if (t.cc_mode == RFSR_CC_RME) CK(launch_rme_field(t, e->stream));
        CK(launch_cc_project(t, e->stream));
    }
    if (prof) CK(cudaEventRecord(sl.phase[3], e->stream));
    CK(launch_fsr(t, e->stream));
    if (prof) CK(cudaEventRecord(sl.phase[4], e->stream));
    CK(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    return RFSR_OK;
}

// device memory of the engine itself (batch tables): the caller's allocator when given
cudaError_t engine_alloc(rfsr_engine *e, void **p, size_t n)
{
    if (e->cfg.dev_alloc) {
        *p = e->cfg.dev_alloc(n, e->cfg.alloc_ctx);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, n);
}

void engine_free(rfsr_engine *e, void *p)
{
    if (e->cfg.dev_free) e->cfg.dev_free(p, e->cfg.alloc_ctx);
    else cudaFree(p);
}

// launch the phases of one batch (captured into a graph, or directly); ph (tuning only): events
// recorded before / after ME and before / after FSR
cudaError_t launch_batch_phases(BatchDesc *d, int T, bool rme, bool trace, const BatchShape &sh,
                                cudaStream_t st, cudaEvent_t *ph = nullptr)
{
    cudaError_t e = launch_batch_prologue(d, st);
    if (e == cudaSuccess) e = launch_ingest_batched(d, st);
    if (e == cudaSuccess && ph) e = cudaEventRecord(ph[0], st);
    if (e == cudaSuccess) e = launch_me_batched(d, T, sh.me_warps, sh.me_box, st);
    if (e == cudaSuccess && ph) e = cudaEventRecord(ph[1], st);
    if (e == cudaSuccess && rme) e = launch_rme_batched(d, T, st);
    if (e == cudaSuccess) e = launch_cc_batched(d, T, st);
    if (e == cudaSuccess && ph) e = cudaEventRecord(ph[2], st);
    if (e == cudaSuccess) e = launch_fsr_batched(d, sh.fsr_blocks, trace, st);
    if (e == cudaSuccess && ph) e = cudaEventRecord(ph[3], st);
    return e;
}

// fold a finished tuning measurement of set into the tuner and decide once every candidate is
// measured (engine lock held; the set's batch must be complete)
int harvest_tuning(rfsr_engine *e, BatchSet &set)
{
    if (!set.tune_pending) return RFSR_OK;
    set.tune_pending = false;
    Tuner &tu = e->tune;
    float me_ms = 0.f, fsr_ms = 0.f;
    CK(cudaEventElapsedTime(&me_ms, set.ph[0], set.ph[1]));
    CK(cudaEventElapsedTime(&fsr_ms, set.ph[2], set.ph[3]));
    if (set.tune_me >= 0 && set.me_units > 0) {
        tu.me_ns[set.tune_me] += 1e6 * me_ms / set.me_units;
        tu.me_n[set.tune_me]++;
    }
    if (set.tune_fsr >= 0 && set.fsr_units > 0) {
        tu.fsr_ns[set.tune_fsr] += 1e6 * fsr_ms / set.fsr_units;
        tu.fsr_n[set.tune_fsr]++;
    }
    tu.measured++;
    if (!tu.active) return RFSR_OK;
    bool all = true;
    for (int i = 0; i < Tuner::kFsr; ++i) all = all && tu.fsr_n[i] >= Tuner::kSamples;
    const bool me_seen = tu.me_n[0] + tu.me_n[1] > 0;    // no T = 9 work: ME keeps its default
    for (int i = 0; i < Tuner::kMe && me_seen; ++i) all = all && tu.me_n[i] >= Tuner::kSamples;
    if (!all && tu.steps < Tuner::kMaxSteps) return RFSR_OK;
    auto pick = [](const double *ns, const int *cnt, const int *cand, int n, int dflt) {
        int best = dflt;
        double bv = -1.0;
        for (int i = 0; i < n; ++i)
            if (cnt[i] > 0 && (bv < 0.0 || ns[i] / cnt[i] < bv)) {
                bv = ns[i] / cnt[i];
                best = cand[i];
            }
        return best;
    };
    const int me = pick(tu.me_ns, tu.me_n, Tuner::me_cand, Tuner::kMe,
                        e->shape.me_box ? 0 : e->shape.me_warps);
    e->shape.me_box = me == 0 ? 1 : 0;
    e->shape.me_warps = me == 0 ? 8 : me;
    e->shape.fsr_blocks = pick(tu.fsr_ns, tu.fsr_n, Tuner::fsr_cand, Tuner::kFsr, e->shape.fsr_blocks);
    tu.active = false;
    return RFSR_OK;
}

// one batched step over at most kMaxBatch streams sharing one template size (engine lock held).
// Returns the number of frames launched.
int step_batch_locked(rfsr_engine *e)
{
    if (e->staged <= 0) return 0;
    BatchSet &set = e->sets[e->next_set];
    if (set.used) {                                  // its previous batch must be done
        cudaError_t er = cudaEventSynchronize(set.done);
        if (er != cudaSuccess) return cuda_fail(er, "cudaEventSynchronize");
        const int rc = harvest_tuning(e, set);
        if (rc != RFSR_OK) return rc;
    }
    BatchDesc *bd = set.h;
    int T = -1, n = 0;
    bool rme = false, trace = false;
    std::vector<std::pair<rfsr_stream *, int>> taken;
    for (rfsr_stream *s : e->streams) {
        if (!s->live || s->launched >= s->pushed || n >= kMaxBatch) continue;
        if (T < 0) T = s->cfg.template_size;
        if (s->cfg.template_size != T) continue;
        const int si = (int)(s->launched % (long long)s->slots.size());
        Slot &sl = s->slots[si];
        FrameTask &t = bd->task[n];
        prepare_frame(s, si, sl.in_smp, sl.in_msk, t);
        t.status_out = sl.h_status_dev;
        if (sl.host_push) t.out_u8 = sl.h_out_dev;
        rme = rme || t.cc_mode == RFSR_CC_RME;
        trace = trace || t.fsr_sel != nullptr;
        taken.emplace_back(s, si);
        ++n;
    }
    if (n == 0) return 0;
    for (auto &p : taken) {                          // device pushes: their producers' work first
        Slot &sl = p.first->slots[p.second];
        if (sl.wait_ready) {
            CK(cudaStreamWaitEvent(e->stream, sl.ready, 0));
            sl.wait_ready = false;
        }
    }
    // tile shape of this step: a tuning candidate while the tuner measures, else the engine's
    Tuner &tu = e->tune;
    const bool tuning = tu.active;
    BatchShape sh = e->shape;
    int cme = -1, cfsr = -1;
    if (tuning) {
        cfsr = tu.steps % Tuner::kFsr;
        sh.fsr_blocks = Tuner::fsr_cand[cfsr];
        if (T == 9) {
            cme = tu.steps % Tuner::kMe;
            sh.me_warps = Tuner::me_cand[cme] ? Tuner::me_cand[cme] : 8;
            sh.me_box = Tuner::me_cand[cme] ? 0 : 1;
        }
    }
    bd->ntasks = n;
    int tot[kPhases] = {0, 0, 0, 0, 0};
    double me_units = 0, fsr_units = 0;
    for (int i = 0; i < n; ++i) {
        const FrameTask &t = bd->task[i];
        // a stream with concealed weighting > 0 gets no FSR tiles: its blocks run as wavefronts
        // after the batch (below)
        const bool conc = t.fsr_concealed > 0.f;
        const int c[kPhases] = {tiles_ingest(t), tiles_me(t, sh.me_warps, sh.me_box), tiles_rme(t), tiles_cc(t),
                                conc ? 0 : tiles_fsr(t, sh.fsr_blocks)};
        for (int p = 0; p < kPhases; ++p) {
            bd->off[p][i] = tot[p];
            tot[p] += c[p];
        }
        me_units += (double)t.H * t.W * t.K;
        if (!conc) fsr_units += (double)((t.H + kFsrB - 1) / kFsrB) * ((t.W + kFsrB - 1) / kFsrB);
    }
    for (int p = 0; p < kPhases; ++p) {
        bd->off[p][n] = tot[p];
        bd->ntiles[p] = tot[p];
        bd->queue[p] = 0;
    }
    const bool prof = e->cfg.profile != 0;
    if (prof) CK(cudaEventRecord(set.t0, e->stream));
    const int key = 4 * T + (trace ? 2 : 0) + (rme ? 1 : 0);
    bool launched = false;
    if (e->graphs_ok && !tuning) {
        auto it = set.graphs.find(key);
        if (it == set.graphs.end()) {
            const long long before = launches();
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            cudaError_t er = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
            if (er == cudaSuccess) {
                cudaError_t er2 = cudaMemcpyAsync(set.d, set.h, sizeof(BatchDesc),
                                                  cudaMemcpyHostToDevice, e->stream);
                if (er2 == cudaSuccess) er2 = launch_batch_phases(set.d, T, rme, trace, sh, e->stream);
                er = cudaStreamEndCapture(e->stream, &g);
                if (er == cudaSuccess) er = er2;
            }
            if (er == cudaSuccess) er = cudaGraphInstantiate(&ex, g, 0);
            if (g) cudaGraphDestroy(g);
            const int nk = (int)(launches() - before);
            count_launch(-nk);                       // counted again at every replay
            if (er == cudaSuccess) {
                it = set.graphs.emplace(key, ex).first;
                set.graph_kernels[key] = nk;
            } else {
                e->graphs_ok = false;                // fall back to direct launches
                cudaGetLastError();
            }
        }
        if (e->graphs_ok) {
            CK(cudaGraphLaunch(it->second, e->stream));
            count_launch(set.graph_kernels[key]);
            launched = true;
        }
    }
    if (!launched) {
        CK(cudaMemcpyAsync(set.d, set.h, sizeof(BatchDesc), cudaMemcpyHostToDevice, e->stream));
        CK(launch_batch_phases(set.d, T, rme, trace, sh, e->stream, tuning ? set.ph : nullptr));
    }
    // concealed weighting > 0 (Sec. 4 sets it to 0; the original FSR): each such stream's FSR runs
    // as its own wavefront launches, on the same stream right after the batch's checks and FSR
    for (int i = 0; i < n; ++i)
        if (bd->task[i].fsr_concealed > 0.f) CK(launch_fsr(bd->task[i], e->stream));
    if (tuning) {
        set.tune_pending = true;
        set.tune_me = cme;
        set.tune_fsr = cfsr;
        set.me_units = me_units;
        set.fsr_units = fsr_units;
        tu.steps++;
    }
    if (prof) CK(cudaEventRecord(set.t1, e->stream));
    CK(cudaEventRecord(set.done, e->stream));
    set.used = true;
    for (auto &p : taken) {
        CK(cudaEventRecord(p.first->slots[p.second].done, e->stream));
        p.first->launched++;
        e->staged--;
    }
    e->last_batch_set = e->next_set;
    e->last_batch_frames = n;
    e->batches++;
    e->next_set ^= 1;
    return n;
}

void serve_loop(rfsr_engine *e)
{
    cudaSetDevice(e->cfg.device);
    std::unique_lock<std::mutex> lk(e->mu);
    while (!e->stop) {
        e->cv.wait(lk, [&] { return e->stop || e->staged > 0; });
        if (e->stop) break;
        if (step_batch_locked(e) < 0) {
            // a CUDA error: leave the frames to time out in rfsr_get_frame and back off
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::milliseconds(1));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

void rfsr_engine_config_default(rfsr_engine_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->device = 0;
    c->max_inflight = 4;
    c->autotune = 1;
}

void rfsr_stream_config_default(rfsr_stream_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->height = 720;
    c->width = 1280;
    c->mask_type = RFSR_MASK_DYNAMIC;
    c->cc_mode = RFSR_CC_NNC_FRMC;
    c->num_refs = 3;
    c->template_size = 9;
    c->search_radius = 8;
    c->check_radius = 8;
    c->fsr_iterations = 100;
    c->fsr_rho = 0.7f;
    c->fsr_gamma = 0.5f;
    c->fsr_proj_weight = 1.0f;
    c->fsr_overwrite_projected = 0;
    c->keep_f32 = 0;
}

const char *rfsr_last_error(void) { return g_err.c_str(); }

long long rfsr_kernel_launches(void) { return rfsr::launches(); }

int rfsr_fused_schedule(int height, int width, int num_refs, int grid, uint32_t *items, int capacity)
{
    if (height < 16 || width < 16 || height > 8192 || width > 8192 || num_refs < 1 ||
        num_refs > kMaxRefs || grid < 1 || capacity < 0)
        return fail(RFSR_EINVAL, "fused_schedule: bad size, past frames or grid");
    const int n = mecc_schedule(height, width, num_refs, grid, nullptr);
    if (items && capacity >= n) mecc_schedule(height, width, num_refs, grid, items);
    return n;
}

int rfsr_engine_create(const rfsr_engine_config *cfg, rfsr_engine **out)
{
    if (!cfg || !out) return fail(RFSR_EINVAL, "engine_create: NULL argument");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (cfg->device < 0 || cfg->device >= ndev) return fail(RFSR_EINVAL, "engine_create: no such device");
    if (cfg->max_inflight < 0 || cfg->max_inflight > 64)
        return fail(RFSR_EINVAL, "engine_create: max_inflight out of range");
    if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr))
        return fail(RFSR_EINVAL, "engine_create: set both dev_alloc and dev_free, or neither");
    CK(cudaSetDevice(cfg->device));
    auto *e = new rfsr_engine();
    e->cfg = *cfg;
    if (e->cfg.max_inflight == 0) e->cfg.max_inflight = 4;
    auto bail = [&](cudaError_t er, const char *what) {
        for (auto &set : e->sets) {
            if (set.h) cudaFreeHost(set.h);
            if (set.d) engine_free(e, set.d);
            if (set.done) cudaEventDestroy(set.done);
            if (set.t0) cudaEventDestroy(set.t0);
            if (set.t1) cudaEventDestroy(set.t1);
            for (auto &ev : set.ph)
                if (ev) cudaEventDestroy(ev);
        }
        if (e->own_stream) cudaStreamDestroy(e->stream);
        delete e;
        return cuda_fail(er, what);
    };
    if (cfg->cuda_stream) {
        e->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        cudaError_t err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) return bail(err, "cudaStreamCreateWithFlags");
        e->own_stream = true;
    }
    cudaError_t ie = init_fsr(cfg->device);
    if (ie != cudaSuccess) return bail(ie, "FSR set-up");
    ie = init_cc(cfg->device);
    if (ie != cudaSuccess) return bail(ie, "check set-up");
    ie = init_me(cfg->device);
    if (ie != cudaSuccess) return bail(ie, "ME set-up");
    if (batched(e)) {
        for (auto &set : e->sets) {
            cudaError_t er = cudaHostAlloc((void **)&set.h, sizeof(BatchDesc), cudaHostAllocPortable);
            if (er == cudaSuccess) er = engine_alloc(e, (void **)&set.d, sizeof(BatchDesc));
            if (er == cudaSuccess) er = cudaEventCreateWithFlags(&set.done, cudaEventDisableTiming);
            if (er == cudaSuccess) er = cudaEventCreate(&set.t0);
            if (er == cudaSuccess) er = cudaEventCreate(&set.t1);
            for (auto &ev : set.ph)
                if (er == cudaSuccess) er = cudaEventCreate(&ev);
            if (er != cudaSuccess) return bail(er, "batch buffers");
            std::memset(set.h, 0, sizeof(BatchDesc));
        }
    }
    size_t fr = 0, tot = 0;
    cudaError_t er = cudaMemGetInfo(&fr, &tot);
    if (er != cudaSuccess) return bail(er, "cudaMemGetInfo");
    e->budget = cfg->memory_budget ? cfg->memory_budget : (size_t)(0.8 * (double)fr);
    e->tune.active = batched(e) && cfg->autotune != 0;
    if (cfg->serve) e->server = std::thread(serve_loop, e);
    *out = e;
    return RFSR_OK;
}

int rfsr_engine_sync(rfsr_engine *e, int timeout_ms)
{
    if (!e) return fail(RFSR_EINVAL, "engine_sync: NULL engine");
    CK(cudaSetDevice(e->cfg.device));
    const auto t0 = Clock::now();
    if (batched(e)) {                                // wait until every staged frame is launched
        for (;;) {
            {
                std::lock_guard<std::mutex> g(e->mu);
                if (e->staged == 0) break;
                if (!e->cfg.serve) return fail(RFSR_ESTATE, "engine_sync: frames staged; call rfsr_engine_step");
            }
            if (timeout_ms >= 0 &&
                std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() >= timeout_ms)
                return fail(RFSR_ETIMEDOUT, "engine_sync: staged frames not launched within timeout");
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t err;
    {
        std::lock_guard<std::mutex> g(e->mu);
        err = cudaEventRecord(ev, e->stream);
    }
    if (err != cudaSuccess) {
        cudaEventDestroy(ev);
        return cuda_fail(err, "cudaEventRecord");
    }
    int rc = wait_event(ev, timeout_ms, t0);
    cudaEventDestroy(ev);
    return rc;
}

int rfsr_destroy(rfsr_stream *s);

int rfsr_engine_destroy(rfsr_engine *e)
{
    if (!e) return fail(RFSR_EINVAL, "engine_destroy: NULL engine");
    cudaSetDevice(e->cfg.device);
    if (e->server.joinable()) {
        {
            std::lock_guard<std::mutex> g(e->mu);
            e->stop = true;
        }
        e->cv.notify_all();
        e->server.join();
        e->cfg.serve = 0;                           // streams left are stepped by rfsr_destroy
    }
    cudaStreamSynchronize(e->stream);
    std::vector<rfsr_stream *> ss;
    {
        std::lock_guard<std::mutex> g(e->mu);
        ss = e->streams;
    }
    for (auto *s : ss) rfsr_destroy(s);
    for (auto &set : e->sets) {
        for (auto &kv : set.graphs) cudaGraphExecDestroy(kv.second);
        if (set.h) cudaFreeHost(set.h);
        if (set.d) engine_free(e, set.d);
        if (set.done) cudaEventDestroy(set.done);
        if (set.t0) cudaEventDestroy(set.t0);
        if (set.t1) cudaEventDestroy(set.t1);
        for (auto &ev : set.ph)
            if (ev) cudaEventDestroy(ev);
    }
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
    return RFSR_OK;
}

int rfsr_engine_step(rfsr_engine *e)
{
    if (!e) return fail(RFSR_EINVAL, "engine_step: NULL engine");
    if (!batched(e)) return fail(RFSR_ESTATE, "engine_step: engine is not batched");
    CK(cudaSetDevice(e->cfg.device));
    std::lock_guard<std::mutex> g(e->mu);
    int total = 0;
    for (;;) {
        const int n = step_batch_locked(e);
        if (n < 0) return n;
        if (n == 0) break;
        total += n;
    }
    return total;
}

int rfsr_engine_last_step_ms(rfsr_engine *e, float *ms, int *frames)
{
    if (!e || !ms) return fail(RFSR_EINVAL, "engine_last_step_ms: NULL argument");
    if (!batched(e) || !e->cfg.profile)
        return fail(RFSR_ESTATE, "engine_last_step_ms: needs a batched engine with profile = 1");
    BatchSet *set;
    int nf;
    {
        std::lock_guard<std::mutex> g(e->mu);
        if (e->last_batch_set < 0) return fail(RFSR_ESTATE, "engine_last_step_ms: no batch launched");
        set = &e->sets[e->last_batch_set];
        nf = e->last_batch_frames;
    }
    CK(cudaSetDevice(e->cfg.device));
    CK(cudaEventSynchronize(set->t1));
    CK(cudaEventElapsedTime(ms, set->t0, set->t1));
    if (frames) *frames = nf;
    return RFSR_OK;
}

int rfsr_engine_set_shape(rfsr_engine *e, const rfsr_batch_shape *shape)
{
    if (!e || !shape) return fail(RFSR_EINVAL, "engine_set_shape: NULL argument");
    if (!batched(e)) return fail(RFSR_ESTATE, "engine_set_shape: engine is not batched");
    BatchShape sh;
    sh.me_warps = shape->me_tile_rows / 8;
    sh.me_box = shape->me_variant;
    sh.fsr_blocks = shape->fsr_blocks;
    if ((shape->me_tile_rows != 32 && shape->me_tile_rows != 64) || !shape_valid(sh))
        return fail(RFSR_EINVAL, "engine_set_shape: me_tile_rows must be 32 or 64, me_variant 0 or 1, "
                                 "fsr_blocks 2, 4 or 8");
    CK(cudaSetDevice(e->cfg.device));
    std::lock_guard<std::mutex> g(e->mu);
    for (auto &set : e->sets) {                      // graphs of the old shape go
        if (set.used) CK(cudaEventSynchronize(set.done));
        const int rc = harvest_tuning(e, set);
        if (rc != RFSR_OK) return rc;
        for (auto &kv : set.graphs) cudaGraphExecDestroy(kv.second);
        set.graphs.clear();
        set.graph_kernels.clear();
    }
    e->shape = sh;
    e->tune.active = false;
    return RFSR_OK;
}

int rfsr_engine_get_tuning(rfsr_engine *e, rfsr_tuning *out)
{
    if (!e || !out) return fail(RFSR_EINVAL, "engine_get_tuning: NULL argument");
    if (!batched(e)) return fail(RFSR_ESTATE, "engine_get_tuning: engine is not batched");
    CK(cudaSetDevice(e->cfg.device));
    std::lock_guard<std::mutex> g(e->mu);
    for (auto &set : e->sets)                        // fold in measurements that have finished
        if (set.tune_pending && cudaEventQuery(set.done) == cudaSuccess) {
            const int rc = harvest_tuning(e, set);
            if (rc != RFSR_OK) return rc;
        }
    const Tuner &tu = e->tune;
    std::memset(out, 0, sizeof(*out));
    out->tuned = tu.active ? 0 : 1;
    out->steps = tu.measured;
    out->shape.me_tile_rows = 8 * e->shape.me_warps;
    out->shape.me_variant = e->shape.me_box;
    out->shape.fsr_blocks = e->shape.fsr_blocks;
    for (int i = 0; i < Tuner::kMe; ++i) out->me_ns[i] = tu.me_n[i] ? (float)(tu.me_ns[i] / tu.me_n[i]) : 0.f;
    for (int i = 0; i < Tuner::kFsr; ++i)
        out->fsr_ns[i] = tu.fsr_n[i] ? (float)(tu.fsr_ns[i] / tu.fsr_n[i]) : 0.f;
    return RFSR_OK;
}

static int check_stream_config(const rfsr_stream_config *c)
{
    if (c->height < 16 || c->width < 16 || c->height > 8192 || c->width > 8192 ||
        (c->height & 1) || (c->width & 1))
        return fail(RFSR_EINVAL, "stream config: height / width must be even, in [16, 8192]");
    if (c->cc_mode < 0 || c->cc_mode > 5) return fail(RFSR_EINVAL, "stream config: cc_mode");
    if (c->num_refs < 0 || c->num_refs > kMaxRefs) return fail(RFSR_EINVAL, "stream config: num_refs");
    if (c->template_size < 1 || c->template_size > 2 * kMaxHalf + 1 || !(c->template_size & 1))
        return fail(RFSR_EINVAL, "stream config: template_size must be odd, 1..11");
    if (c->search_radius < 1 || c->search_radius > kMaxRadius)
        return fail(RFSR_EINVAL, "stream config: search_radius must be 1..9");
    if (c->check_radius < 1 || c->check_radius > kMaxRadius)
        return fail(RFSR_EINVAL, "stream config: check_radius must be 1..9");
    if (c->fsr_iterations < 0 || c->fsr_iterations > 100000)
        return fail(RFSR_EINVAL, "stream config: fsr_iterations");
    if (!(c->fsr_rho > 0.f && c->fsr_rho <= 1.f)) return fail(RFSR_EINVAL, "stream config: fsr_rho");
    if (!(c->fsr_gamma > 0.f && c->fsr_gamma <= 2.f)) return fail(RFSR_EINVAL, "stream config: fsr_gamma");
    if (!(c->fsr_proj_weight >= 0.f)) return fail(RFSR_EINVAL, "stream config: fsr_proj_weight");
    if (!(c->fsr_concealed_weight >= 0.f && c->fsr_concealed_weight <= 1e6f))
        return fail(RFSR_EINVAL, "stream config: fsr_concealed_weight must be >= 0");
    if (c->fsr_trace != 0 && c->fsr_trace != 1) return fail(RFSR_EINVAL, "stream config: fsr_trace must be 0 or 1");
    if (c->me_predict_radius < 0 || c->me_predict_radius > 2 * kMaxRadius)
        return fail(RFSR_EINVAL, "stream config: me_predict_radius must be 0..18");
    if (c->me_predict_radius > 0 && c->template_size != 9)
        return fail(RFSR_EINVAL, "stream config: me_predict_radius needs template_size 9");
    return RFSR_OK;
}

// the process-wide engine used when a stream call passes NULL (created once, on the device that
// is current for the first such call; it lives until the process ends)
static rfsr_engine *default_engine(int *rc)
{
    static std::mutex m;
    static rfsr_engine *eng = nullptr;
    std::lock_guard<std::mutex> g(m);
    *rc = RFSR_OK;
    if (!eng) {
        rfsr_engine_config c;
        rfsr_engine_config_default(&c);
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            *rc = fail(RFSR_EDEVICE, "default engine: no CUDA device");
            return nullptr;
        }
        c.device = dev;
        *rc = rfsr_engine_create(&c, &eng);
        if (*rc) eng = nullptr;
    }
    return eng;
}

int rfsr_create_stream(rfsr_engine *e, const rfsr_stream_config *cfg, rfsr_stream **out)
{
    if (!cfg || !out) return fail(RFSR_EINVAL, "create_stream: NULL argument");
    if (!e) {
        int rc = 0;
        e = default_engine(&rc);
        if (!e) return rc;
    }
    int rc = check_stream_config(cfg);
    if (rc) return rc;
    if (cfg->me_predict_radius > 0 && batched(e))
        return fail(RFSR_EINVAL, "create_stream: me_predict_radius needs an unbatched engine");
    CK(cudaSetDevice(e->cfg.device));
    auto *s = new rfsr_stream();
    s->eng = e;
    s->cfg = *cfg;
    s->H = cfg->height;
    s->W = cfg->width;
    s->K = cfg->num_refs;
    s->need = stream_need(cfg, e->cfg.max_inflight, fused_me_cc(e->cfg, cfg));
    std::lock_guard<std::mutex> g(e->mu);
    if (s->need > e->budget) {
        delete s;
        return fail(RFSR_ENOMEM, "create_stream: the stream alone exceeds the engine memory budget");
    }
    if (!e->queued.empty() || e->used + s->need > e->budget) {
        e->queued.push_back(s);
        e->streams.push_back(s);
        *out = s;
        return fail(RFSR_EAGAIN, "create_stream: queued until device memory frees up");
    }
    e->used += s->need;
    rc = admit(s);
    if (rc) {
        e->used -= s->need;
        delete s;
        return rc;
    }
    e->streams.push_back(s);
    *out = s;
    return RFSR_OK;
}

static int push_common(rfsr_stream *s)
{
    if (!s->live) return fail(RFSR_EAGAIN, "push_frame: stream is queued for admission");
    if (s->poisoned) return fail(RFSR_ESTATE, "push_frame: stream had a bad mask; reset it with rfsr_set_history");
    if (s->pushed - s->collected >= (long long)s->slots.size())
        return fail(RFSR_EBUSY, "push_frame: in-flight limit reached, collect frames first");
    return RFSR_OK;
}

int rfsr_push_frame(rfsr_stream *s, const uint8_t *samples, const uint8_t *mask)
{
    if (!s || !samples || !mask) return fail(RFSR_EINVAL, "push_frame: NULL argument");
    if (!mask_ok(mask, s->H, s->W)) return fail(RFSR_EMASK, "push_frame: not a quarter-sampling mask");
    rfsr_engine *e = s->eng;
    CK(cudaSetDevice(e->cfg.device));
    const size_t HW = (size_t)s->H * s->W;
    std::unique_lock<std::mutex> lk(e->mu);
    int rc = push_common(s);
    if (rc) return rc;
    const int si = (int)(s->pushed % (long long)s->slots.size());
    Slot &sl = s->slots[si];
    std::memcpy(sl.h_in, samples, HW);
    std::memcpy(sl.h_in + HW, mask, HW);
    sl.host_push = true;
    sl.wait_ready = false;
    if (batched(e)) {
        sl.in_smp = sl.h_in_dev;
        sl.in_msk = sl.h_in_dev + HW;
        s->pushed++;
        e->staged++;
        lk.unlock();
        e->cv.notify_one();
        return RFSR_OK;
    }
    cudaStream_t st = e->stream;
    CK(cudaMemcpyAsync(sl.d_in, sl.h_in, 2 * HW, cudaMemcpyHostToDevice, st));
    rc = enqueue_step(s, si, sl.d_in, sl.d_in + HW);
    if (rc) return rc;
    CK(cudaMemcpyAsync(sl.h_out, sl.d_out, HW, cudaMemcpyDeviceToHost, st));
    if (sl.h_out32) CK(cudaMemcpyAsync(sl.h_out32, sl.d_out32, 4 * HW, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(sl.done, st));
    s->pushed++;
    s->launched++;
    return RFSR_OK;
}

int rfsr_push_frame_device(rfsr_stream *s, const uint8_t *d_samples, const uint8_t *d_mask,
                           void *producer_stream)
{
    if (!s || !d_samples || !d_mask) return fail(RFSR_EINVAL, "push_frame: NULL argument");
    if (((uintptr_t)d_samples | (uintptr_t)d_mask) & 1u)
        return fail(RFSR_EINVAL, "push_frame_device: buffers must be 2-byte aligned");
    rfsr_engine *e = s->eng;
    CK(cudaSetDevice(e->cfg.device));
    std::unique_lock<std::mutex> lk(e->mu);
    int rc = push_common(s);
    if (rc) return rc;
    const int si = (int)(s->pushed % (long long)s->slots.size());
    Slot &sl = s->slots[si];
    sl.host_push = false;
    // the engine's stream waits for the producer's work on these buffers (no host wait)
    const cudaStream_t prod = (cudaStream_t)producer_stream;
    sl.wait_ready = prod != nullptr && prod != e->stream;
    if (sl.wait_ready) CK(cudaEventRecord(sl.ready, prod));
    if (batched(e)) {
        sl.in_smp = d_samples;
        sl.in_msk = d_mask;
        s->pushed++;
        e->staged++;
        lk.unlock();
        e->cv.notify_one();
        return RFSR_OK;
    }
    if (sl.wait_ready) {
        CK(cudaStreamWaitEvent(e->stream, sl.ready, 0));
        sl.wait_ready = false;
    }
    rc = enqueue_step(s, si, d_samples, d_mask);
    if (rc) return rc;
    CK(cudaEventRecord(sl.done, e->stream));
    s->pushed++;
    s->launched++;
    return RFSR_OK;
}

// wait (bounded) until the oldest uncollected frame is launched and done
static int collect(rfsr_stream *s, int timeout_ms, Slot **out)
{
    rfsr_engine *e = s->eng;
    const auto t0 = Clock::now();
    int si;
    {
        std::lock_guard<std::mutex> g(e->mu);
        if (s->collected >= s->pushed) return fail(RFSR_ESTATE, "get_frame: no frame pushed");
        si = (int)(s->collected % (long long)s->slots.size());
    }
    for (int spins = 0;; ++spins) {                 // batched engines: wait for its launch
        {
            std::lock_guard<std::mutex> g(e->mu);
            if (s->launched > s->collected) break;
        }
        if (timeout_ms >= 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() >= timeout_ms)
            return fail(RFSR_ETIMEDOUT,
                        "frame not launched within timeout (batched engine: call rfsr_engine_step)");
        if (spins < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    Slot &sl = s->slots[si];
    int rc = wait_event(sl.done, timeout_ms, t0);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(e->mu);
        s->collected++;
    }
    const int st = *(volatile int *)sl.h_status;
    if (st & kStatusBadMask) {
        s->poisoned = true;
        return fail(RFSR_EMASK, "get_frame: the frame's device mask is not a quarter-sampling mask");
    }
    if (st & kStatusPoisoned) {
        s->poisoned = true;
        return fail(RFSR_ESTATE, "get_frame: an earlier frame of the stream had a bad mask");
    }
    if (st & kStatusWaitTimeout) {                   // the frame's checks and FSR did not run
        s->poisoned = true;
        return fail(RFSR_EDEVICE, "get_frame: a wait of the fused ME + checks launch ran out; "
                                  "reset the stream with rfsr_set_history");
    }
    *out = &sl;
    return RFSR_OK;
}

int rfsr_get_frame(rfsr_stream *s, uint8_t *out_u8, float *out_f32, int timeout_ms)
{
    if (!s) return fail(RFSR_EINVAL, "get_frame: NULL stream");
    if (out_f32 && !s->cfg.keep_f32) return fail(RFSR_EINVAL, "get_frame: out_f32 needs keep_f32");
    CK(cudaSetDevice(s->eng->cfg.device));
    Slot *sl = nullptr;
    int rc = collect(s, timeout_ms, &sl);
    if (rc) return rc;
    const size_t HW = (size_t)s->H * s->W;
    if (sl->host_push) {
        if (out_u8) std::memcpy(out_u8, sl->h_out, HW);
        if (out_f32) {
            if (batched(s->eng)) CK(cudaMemcpy(out_f32, sl->d_out32, 4 * HW, cudaMemcpyDeviceToHost));
            else std::memcpy(out_f32, sl->h_out32, 4 * HW);
        }
    } else {
        if (out_u8) CK(cudaMemcpy(out_u8, sl->d_out, HW, cudaMemcpyDeviceToHost));
        if (out_f32) CK(cudaMemcpy(out_f32, sl->d_out32, 4 * HW, cudaMemcpyDeviceToHost));
    }
    return RFSR_OK;
}

int rfsr_get_frame_device(rfsr_stream *s, uint8_t *d_out_u8, float *d_out_f32, int timeout_ms)
{
    if (!s) return fail(RFSR_EINVAL, "get_frame_device: NULL stream");
    if (d_out_f32 && !s->cfg.keep_f32) return fail(RFSR_EINVAL, "get_frame_device: out_f32 needs keep_f32");
    rfsr_engine *e = s->eng;
    CK(cudaSetDevice(e->cfg.device));
    Slot *sl = nullptr;
    int rc = collect(s, timeout_ms, &sl);
    if (rc) return rc;
    const size_t HW = (size_t)s->H * s->W;
    if (!d_out_u8 && !d_out_f32) return RFSR_OK;
    const uint8_t *src = (sl->host_push && batched(e)) ? sl->h_out_dev : sl->d_out;
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    {
        std::lock_guard<std::mutex> g(e->mu);
        if (d_out_u8) CK(cudaMemcpyAsync(d_out_u8, src, HW, cudaMemcpyDeviceToDevice, e->stream));
        if (d_out_f32) CK(cudaMemcpyAsync(d_out_f32, sl->d_out32, 4 * HW, cudaMemcpyDeviceToDevice, e->stream));
        CK(cudaEventRecord(ev, e->stream));
    }
    rc = wait_event(ev, -1);
    cudaEventDestroy(ev);
    return rc;
}

int rfsr_destroy(rfsr_stream *s)
{
    if (!s) return fail(RFSR_EINVAL, "destroy: NULL stream");
    rfsr_engine *e = s->eng;
    cudaSetDevice(e->cfg.device);
    // frames staged in a batched engine are launched first, then every frame in flight ends
    for (;;) {
        std::unique_lock<std::mutex> lk(e->mu);
        if (s->launched >= s->pushed) break;
        if (!e->cfg.serve) {
            if (step_batch_locked(e) <= 0) break;   // (a CUDA error leaves nothing to wait for)
            continue;
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (auto &sl : s->slots)
        if (sl.done) cudaEventSynchronize(sl.done);
    std::lock_guard<std::mutex> g(e->mu);
    const bool was_live = s->live;
    s->release();
    e->streams.erase(std::remove(e->streams.begin(), e->streams.end(), s), e->streams.end());
    e->queued.erase(std::remove(e->queued.begin(), e->queued.end(), s), e->queued.end());
    if (was_live) e->used -= std::min(e->used, s->need);
    delete s;
    admit_queued(e);
    return RFSR_OK;
}

int rfsr_stream_state(rfsr_stream *s)
{
    if (!s) return fail(RFSR_EINVAL, "stream_state: NULL stream");
    std::lock_guard<std::mutex> g(s->eng->mu);
    return s->live ? 1 : 0;
}

int rfsr_stream_get_info(rfsr_stream *s, rfsr_stream_info *info)
{
    if (!s || !info) return fail(RFSR_EINVAL, "stream_get_info: NULL argument");
    std::lock_guard<std::mutex> g(s->eng->mu);
    info->height = s->H;
    info->width = s->W;
    info->live = s->live ? 1 : 0;
    info->frames_pushed = s->pushed;
    info->frames_collected = s->collected;
    info->history_frames = s->hist;
    info->device_bytes = s->bytes;
    return RFSR_OK;
}

// every pushed frame launched and done (batched engines without a server step them here)
static int wait_all(rfsr_stream *s)
{
    rfsr_engine *e = s->eng;
    for (;;) {
        std::unique_lock<std::mutex> lk(e->mu);
        if (s->launched >= s->pushed) break;
        if (!e->cfg.serve) {
            if (step_batch_locked(e) <= 0) return fail(RFSR_EDEVICE, "wait_all: batched step failed");
            continue;
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (auto &sl : s->slots) CK(cudaEventSynchronize(sl.done));
    return RFSR_OK;
}

int rfsr_set_history(rfsr_stream *s, int nrefs, const uint8_t *const *rec,
                     const uint8_t *const *smp, const uint8_t *const *msk)
{
    if (!s) return fail(RFSR_EINVAL, "set_history: NULL stream");
    if (!s->live) return fail(RFSR_EAGAIN, "set_history: stream is queued for admission");
    if (nrefs < 0 || nrefs > s->K) return fail(RFSR_EINVAL, "set_history: nrefs must be in [0, K]");
    if (nrefs > 0 && (!rec || !smp || !msk)) return fail(RFSR_EINVAL, "set_history: NULL arrays");
    for (int k = 0; k < nrefs; ++k)
        if (!rec[k] || !smp[k] || !msk[k]) return fail(RFSR_EINVAL, "set_history: NULL plane");
    CK(cudaSetDevice(s->eng->cfg.device));
    int rc = wait_all(s);
    if (rc) return rc;
    const size_t HW = (size_t)s->H * s->W;
    std::vector<uint8_t> bm(HW), sm(HW);
    const int R1 = s->K + 1;
    for (int k = 1; k <= nrefs; ++k) {
        if (!mask_ok(msk[k - 1], s->H, s->W))
            return fail(RFSR_EMASK, "set_history: not a quarter-sampling mask");
        for (size_t i = 0; i < HW; ++i) {
            bm[i] = msk[k - 1][i] ? 0xff : 0;
            sm[i] = smp[k - 1][i] & bm[i];
        }
        const int rr = ((s->ring_head - k) % R1 + R1) % R1;
        CK(cudaMemcpy(s->ring_rec[rr], rec[k - 1], HW, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(s->ring_smp[rr], sm.data(), HW, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(s->ring_msk[rr], bm.data(), HW, cudaMemcpyHostToDevice));
    }
    std::lock_guard<std::mutex> g(s->eng->mu);
    s->hist = nrefs;
    s->poisoned = false;
    s->last_slot = -1;      // the poison chain restarts
    return RFSR_OK;
}

int rfsr_stream_export(rfsr_stream *s, void *buf, size_t cap, size_t *bytes)
{
    if (!s || !bytes) return fail(RFSR_EINVAL, "stream_export: NULL argument");
    if (!s->live) return fail(RFSR_EAGAIN, "stream_export: stream is queued for admission");
    const size_t HW = (size_t)s->H * s->W;
    int hist;
    long long frames;
    {
        std::lock_guard<std::mutex> g(s->eng->mu);
        if (s->collected != s->pushed)
            return fail(RFSR_ESTATE, "stream_export: collect every pushed frame first");
        if (s->poisoned) return fail(RFSR_ESTATE, "stream_export: the stream had a bad mask");
        hist = s->hist;
        frames = s->pushed;
    }
    const size_t need = sizeof(rfsr_state_header) + (size_t)hist * 3 * HW;
    *bytes = need;
    if (!buf) return RFSR_OK;
    if (cap < need) return fail(RFSR_EINVAL, "stream_export: buffer too small");
    CK(cudaSetDevice(s->eng->cfg.device));
    int rc = wait_all(s);
    if (rc) return rc;
    rfsr_state_header h;
    std::memset(&h, 0, sizeof(h));
    h.magic = RFSR_STATE_MAGIC;
    h.version = RFSR_STATE_VERSION;
    h.bytes = need;
    h.config = s->cfg;
    h.hist = hist;
    h.frames = frames;
    uint8_t *p = static_cast<uint8_t *>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const int R1 = s->K + 1;
    for (int k = 1; k <= hist; ++k) {
        const int rr = ((s->ring_head - k) % R1 + R1) % R1;
        CK(cudaMemcpy(p, s->ring_rec[rr], HW, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(p + HW, s->ring_smp[rr], HW, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(p + 2 * HW, s->ring_msk[rr], HW, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < HW; ++i) p[2 * HW + i] = p[2 * HW + i] ? 1 : 0;   // byte mask -> 0/1
        p += 3 * HW;
    }
    return RFSR_OK;
}

int rfsr_stream_import(rfsr_engine *e, const void *buf, size_t bytes, rfsr_stream **out)
{
    if (!buf || !out) return fail(RFSR_EINVAL, "stream_import: NULL argument");
    if (bytes < sizeof(rfsr_state_header)) return fail(RFSR_EINVAL, "stream_import: buffer too small");
    rfsr_state_header h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != RFSR_STATE_MAGIC || h.version != RFSR_STATE_VERSION)
        return fail(RFSR_EINVAL, "stream_import: not a stream state of this version");
    int rc = check_stream_config(&h.config);
    if (rc) return rc;
    const size_t HW = (size_t)h.config.height * h.config.width;
    if (h.hist < 0 || h.hist > h.config.num_refs || h.bytes != bytes ||
        bytes != sizeof(h) + (size_t)h.hist * 3 * HW)
        return fail(RFSR_EINVAL, "stream_import: inconsistent state size or history");
    rfsr_stream *s = nullptr;
    rc = rfsr_create_stream(e, &h.config, &s);
    if (rc == RFSR_EAGAIN) {
        rfsr_destroy(s);
        return fail(RFSR_EAGAIN, "stream_import: the engine's memory budget is full; retry later");
    }
    if (rc) return rc;
    std::vector<const uint8_t *> rec(h.hist), smp(h.hist), msk(h.hist);
    const uint8_t *p = static_cast<const uint8_t *>(buf) + sizeof(h);
    for (int k = 0; k < h.hist; ++k, p += 3 * HW) {
        rec[k] = p;
        smp[k] = p + HW;
        msk[k] = p + 2 * HW;
    }
    rc = rfsr_set_history(s, h.hist, rec.data(), smp.data(), msk.data());
    if (rc) {
        const std::string msg = g_err;
        rfsr_destroy(s);
        return fail(rc, msg);
    }
    *out = s;
    return RFSR_OK;
}

int rfsr_engine_get_info(rfsr_engine *e, rfsr_engine_info *info)
{
    if (!e || !info) return fail(RFSR_EINVAL, "engine_get_info: NULL argument");
    std::lock_guard<std::mutex> g(e->mu);
    info->device = e->cfg.device;
    info->memory_budget = e->budget;
    info->memory_used = e->used;
    info->streams_queued = (int)e->queued.size();
    info->streams_live = (int)e->streams.size() - info->streams_queued;
    return RFSR_OK;
}

int rfsr_debug_get(rfsr_stream *s, int what, int k, void *dst)
{
    if (!s || !dst) return fail(RFSR_EINVAL, "debug_get: NULL argument");
    if (!s->live || s->pushed == 0) return fail(RFSR_ESTATE, "debug_get: no frame processed");
    CK(cudaSetDevice(s->eng->cfg.device));
    int rc = wait_all(s);
    if (rc) return rc;
    if (s->last_slot < 0) return fail(RFSR_ESTATE, "debug_get: no frame processed");
    const size_t HW = (size_t)s->H * s->W;
    const bool per_ref = what == RFSR_DBG_MV || what == RFSR_DBG_FMV || what == RFSR_DBG_DECISION ||
                         what == RFSR_DBG_RMV;
    if (per_ref && (k < 1 || k > s->last_K)) return fail(RFSR_ESTATE, "debug_get: k outside 1..K of that frame");
    const void *src = nullptr;
    size_t n = 0;
    switch (what) {
    case RFSR_DBG_MV: src = s->mv[k - 1]; n = 2 * HW; break;
    case RFSR_DBG_FMV: src = s->fmv[k - 1]; n = 2 * HW; break;
    case RFSR_DBG_DECISION: src = s->dec[k - 1]; n = HW; break;
    case RFSR_DBG_RMV:
        if (!s->rmv[k - 1]) return fail(RFSR_ESTATE, "debug_get: reverse field exists in RME mode only");
        src = s->rmv[k - 1]; n = 2 * HW; break;
    case RFSR_DBG_PSUM: src = s->psum; n = 2 * HW; break;
    case RFSR_DBG_PCNT: src = s->pcnt; n = HW; break;
    case RFSR_DBG_FSR: {
        const Slot &sl = s->slots[s->last_slot];
        src = sl.d_out32 ? (const void *)sl.d_out32 : (const void *)s->fsr;
        n = 4 * HW;
        break;
    }
    case RFSR_DBG_REC: src = s->ring_rec[s->last_ring]; n = HW; break;
    case RFSR_DBG_FSR_SEL:
        if (!s->fsr_sel) return fail(RFSR_ESTATE, "debug_get: FSR selections are recorded only with fsr_trace = 1");
        src = s->fsr_sel; n = trace_bytes(&s->cfg); break;
    default: return fail(RFSR_EINVAL, "debug_get: unknown plane");
    }
    CK(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost));
    return RFSR_OK;
}

int rfsr_stream_phase_ms(rfsr_stream *s, float ms[4])
{
    if (!s || !ms) return fail(RFSR_EINVAL, "stream_phase_ms: NULL argument");
    if (!s->eng->cfg.profile || batched(s->eng))
        return fail(RFSR_ESTATE, "stream_phase_ms: needs an unbatched engine created with profile = 1");
    if (s->last_slot < 0) return fail(RFSR_ESTATE, "stream_phase_ms: no frame pushed");
    CK(cudaSetDevice(s->eng->cfg.device));
    Slot &sl = s->slots[s->last_slot];
    CK(cudaEventSynchronize(sl.phase[4]));
    for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&ms[i], sl.phase[i], sl.phase[i + 1]));
    return RFSR_OK;
}

static int fsr_device_impl(const rfsr_stream_config *cfg, const uint8_t *d_smp, const uint8_t *d_msk,
                           const uint16_t *d_psum, const uint8_t *d_pcnt, float *d_out_f32,
                           uint8_t *d_out_u8, uint16_t *d_sel, void *cuda_stream)
{
    if (!cfg || !d_smp || !d_msk) return fail(RFSR_EINVAL, "fsr_device: NULL argument");
    if ((d_psum == nullptr) != (d_pcnt == nullptr))
        return fail(RFSR_EINVAL, "fsr_device: psum and pcnt must both be given or both be NULL");
    if (((uintptr_t)d_psum & 1u) || ((uintptr_t)d_out_f32 & 3u))
        return fail(RFSR_EINVAL, "fsr_device: psum must be 2-byte and out_f32 4-byte aligned");
    int rc = check_stream_config(cfg);
    if (rc) return rc;
    if (cfg->fsr_concealed_weight > 0.f && !d_out_f32)
        return fail(RFSR_EINVAL, "fsr_device: concealed weighting > 0 reads d_out_f32, which is NULL");
    // tables and a zero status word, cached per (device, rho)
    static std::mutex mu;
    static std::map<std::pair<int, float>, std::pair<float *, int *>> cache;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    float *tables = nullptr;
    int *zero = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        auto key = std::make_pair(dev, cfg->fsr_rho);
        auto it = cache.find(key);
        if (it == cache.end()) {
            FsrTables tb;
            fill_fsr_tables(tb, cfg->fsr_rho);
            CK(cudaMalloc((void **)&tables, sizeof(tb)));
            CK(cudaMemcpy(tables, &tb, sizeof(tb), cudaMemcpyHostToDevice));
            CK(cudaMalloc((void **)&zero, 64));
            CK(cudaMemset(zero, 0, 64));
            cache[key] = std::make_pair(tables, zero);
        } else {
            tables = it->second.first;
            zero = it->second.second;
        }
    }
    FrameTask t;
    std::memset(&t, 0, sizeof(t));
    t.H = cfg->height;
    t.W = cfg->width;
    t.fsr_iters = cfg->fsr_iterations;
    t.fsr_gamma = cfg->fsr_gamma;
    t.fsr_concealed = cfg->fsr_concealed_weight;
    t.fsr_proj_weight = cfg->fsr_proj_weight;
    t.fsr_overwrite_projected = cfg->fsr_overwrite_projected;
    t.fsr_tables = tables;
    t.cur_smp = const_cast<uint8_t *>(d_smp);
    t.cur_msk = const_cast<uint8_t *>(d_msk);
    t.psum = const_cast<uint16_t *>(d_psum);
    t.pcnt = const_cast<uint8_t *>(d_pcnt);
    t.fsr_out = d_out_f32;
    t.cur_rec = nullptr;
    t.out_u8 = d_out_u8;
    t.status = zero;
    t.fsr_sel = d_sel;
    CK(launch_fsr(t, (cudaStream_t)cuda_stream));
    return RFSR_OK;
}

int rfsr_fsr_device(const rfsr_stream_config *cfg, const uint8_t *d_smp, const uint8_t *d_msk,
                    const uint16_t *d_psum, const uint8_t *d_pcnt, float *d_out_f32,
                    uint8_t *d_out_u8, void *cuda_stream)
{
    return fsr_device_impl(cfg, d_smp, d_msk, d_psum, d_pcnt, d_out_f32, d_out_u8, nullptr,
                           cuda_stream);
}

int rfsr_fsr_device_trace(const rfsr_stream_config *cfg, const uint8_t *d_smp,
                          const uint8_t *d_msk, const uint16_t *d_psum, const uint8_t *d_pcnt,
                          float *d_out_f32, uint8_t *d_out_u8, uint16_t *d_sel, void *cuda_stream)
{
    if (!d_sel || ((uintptr_t)d_sel & 1u))
        return fail(RFSR_EINVAL, "fsr_device_trace: d_sel must be a 2-byte aligned device buffer");
    return fsr_device_impl(cfg, d_smp, d_msk, d_psum, d_pcnt, d_out_f32, d_out_u8, d_sel,
                           cuda_stream);
}

}  // extern "C"
