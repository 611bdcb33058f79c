// noalloc.cu -- motion estimation, consistency checks and projection for one frame without any
// device memory allocation.
//
// Some callers cannot allocate device memory while they run: a real-time loop that has to keep
// its latency free of allocator locks and driver calls, a plugin inside a host application that
// owns all of the GPU's memory and hands out only the buffers it created, or code that must not
// allocate after initialisation at all.  The stream interface allocates its state when a stream
// is created; this entry point instead keeps every intermediate plane of the step (the packed
// current frame, the motion fields, filtered fields, decisions and the status word) in one
// fixed-size array in the library's static device memory.  The caller passes inputs and outputs
// only.  The array exists once per GPU that loads the library and is held until the process ends.
#include <atomic>
#include <cstring>
#include <string>

#include "rfsr.h"
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code its name is a host-side stand-in, not a device address: the
// device address comes from cudaGetSymbolAddress, once per device, with that device current.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::atomic<unsigned char *> g_scratch_addr[kMaxDevices];

size_t up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// bytes of scratch a frame needs: status word, packed sample plane and byte mask, and per past
// frame the raw and filtered motion fields and the decisions (plus the reverse field for RME)
size_t scratch_bytes(int H, int W, int K, int cc_mode)
{
    const size_t HW = (size_t)H * W;
    size_t n = kAlign + 2 * up(HW) + (size_t)K * (2 * up(2 * HW) + up(HW));
    if (cc_mode == RFSR_CC_RME) n += (size_t)K * up(2 * HW);
    return n;
}

int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return RFSR_EDEVICE;
    unsigned char *p = g_scratch_addr[dev].load();
    if (p == nullptr) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_scratch) != cudaSuccess || a == nullptr) return RFSR_EDEVICE;
        p = static_cast<unsigned char *>(a);
        g_scratch_addr[dev].store(p);
    }
    *out = p;
    return RFSR_OK;
}

}  // namespace

}  // namespace rfsr

extern "C" int rfsr_me_cc_project_noalloc(const rfsr_stream_config *cfg, const uint8_t *d_smp,
                                          const uint8_t *d_msk, int nrefs,
                                          const uint8_t *const *d_ref_rec,
                                          const uint8_t *const *d_ref_smp,
                                          const uint8_t *const *d_ref_msk, uint16_t *d_psum,
                                          uint8_t *d_pcnt, uint8_t *d_dec, int *d_status,
                                          void *cuda_stream)
{
    using namespace rfsr;
    const char *what = "me_cc_project_noalloc: ";
    if (!cfg || !d_smp || !d_msk || !d_psum || !d_pcnt)
        return set_error(RFSR_EINVAL, std::string(what) + "NULL argument");
    const int H = cfg->height, W = cfg->width;
    if (H < 16 || W < 16 || H > 8192 || W > 8192 || (H & 1) || (W & 1))
        return set_error(RFSR_EINVAL, std::string(what) + "height / width must be even, in [16, 8192]");
    if (cfg->cc_mode < 0 || cfg->cc_mode > 5) return set_error(RFSR_EINVAL, std::string(what) + "cc_mode");
    if (nrefs < 0 || nrefs > kMaxRefs) return set_error(RFSR_EINVAL, std::string(what) + "nrefs must be 0..3");
    if (nrefs > 0 && (!d_ref_rec || !d_ref_smp || !d_ref_msk))
        return set_error(RFSR_EINVAL, std::string(what) + "NULL reference arrays");
    for (int k = 0; k < nrefs; ++k)
        if (!d_ref_rec[k] || !d_ref_smp[k] || !d_ref_msk[k])
            return set_error(RFSR_EINVAL, std::string(what) + "NULL reference plane");
    if (cfg->template_size < 1 || cfg->template_size > 2 * kMaxHalf + 1 || !(cfg->template_size & 1))
        return set_error(RFSR_EINVAL, std::string(what) + "template_size must be odd, 1..11");
    if (cfg->search_radius < 1 || cfg->search_radius > kMaxRadius ||
        cfg->check_radius < 1 || cfg->check_radius > kMaxRadius)
        return set_error(RFSR_EINVAL, std::string(what) + "search / check radius must be 1..9");
    if (cfg->me_predict_radius < 0 || cfg->me_predict_radius > 2 * kMaxRadius ||
        (cfg->me_predict_radius > 0 && cfg->template_size != 9))
        return set_error(RFSR_EINVAL, std::string(what) + "me_predict_radius must be 0..18 (T = 9 when > 0)");
    if ((((uintptr_t)d_smp | (uintptr_t)d_msk | (uintptr_t)d_psum) & 1u) ||
        ((uintptr_t)d_status & 3u))
        return set_error(RFSR_EINVAL, std::string(what) + "misaligned buffer");
    // the only size limit: the frame's scratch must fit the static array
    const size_t need = scratch_bytes(H, W, nrefs, cfg->cc_mode);
    if (need > kScratchBytes)
        return set_error(RFSR_EINVAL, std::string(what) + "frame needs " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " +
                                          std::to_string(kScratchBytes) + " bytes");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(RFSR_EDEVICE, std::string(what) + "cudaGetDevice");
    unsigned char *base = nullptr;
    if (scratch_address(dev, &base))
        return set_error(RFSR_EDEVICE, std::string(what) + "cudaGetSymbolAddress of the scratch array failed");

    const size_t HW = (size_t)H * W;
    size_t off = 0;
    auto take = [&](size_t n) {
        unsigned char *p = base + off;
        off += up(n);
        return p;
    };
    FrameTask t;
    std::memset(&t, 0, sizeof(t));
    t.H = H;
    t.W = W;
    t.K = nrefs;
    t.T = cfg->template_size;
    t.R = cfg->search_radius;
    t.Rc = cfg->check_radius;
    t.me_pred = cfg->me_predict_radius;
    t.cc_mode = cfg->cc_mode;
    t.status = reinterpret_cast<int *>(take(kAlign));
    t.prev_status = nullptr;
    t.in_smp = d_smp;
    t.in_msk = d_msk;
    t.cur_smp = take(HW);
    t.cur_msk = take(HW);
    for (int k = 0; k < nrefs; ++k) {
        t.ref_rec[k] = d_ref_rec[k];
        t.ref_smp[k] = d_ref_smp[k];
        t.ref_msk[k] = d_ref_msk[k];
        t.mv[k] = reinterpret_cast<int8_t *>(take(2 * HW));
        t.fmv[k] = reinterpret_cast<int8_t *>(take(2 * HW));
        // the check kernel writes the decisions straight into the caller's d_dec when given (it
        // writes nothing when the mask is bad, so d_dec is then left as it was)
        t.dec[k] = take(HW);
        if (d_dec) t.dec[k] = d_dec + (size_t)k * HW;
        if (cfg->cc_mode == RFSR_CC_RME) t.rmv[k] = reinterpret_cast<int8_t *>(take(2 * HW));
    }
    t.psum = d_psum;
    t.pcnt = d_pcnt;

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    auto dev_fail = [&](cudaError_t e, const char *call) {
        return set_error(RFSR_EDEVICE, std::string(what) + call + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    // the array keeps the previous call's contents: the status word must start at zero; every
    // other plane is written in full before it is read
    if ((e = cudaMemsetAsync(t.status, 0, sizeof(int), st)) != cudaSuccess) return dev_fail(e, "cudaMemsetAsync");
    if ((e = launch_ingest(t, st)) != cudaSuccess) return dev_fail(e, "ingest launch");
    if ((e = launch_me(t, st)) != cudaSuccess) return dev_fail(e, "ME launch");
    if (t.cc_mode == RFSR_CC_RME && (e = launch_rme_field(t, st)) != cudaSuccess)
        return dev_fail(e, "RME launch");
    if ((e = launch_cc_project(t, st)) != cudaSuccess) return dev_fail(e, "check launch");
    if (d_status &&
        (e = cudaMemcpyAsync(d_status, t.status, sizeof(int), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return dev_fail(e, "cudaMemcpyAsync");
    return RFSR_OK;
}
