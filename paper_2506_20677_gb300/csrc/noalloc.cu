// Feature extraction for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at the point where they need the
// features of an array: loops whose device memory is fully reserved up front
// by another allocator or pool (a framework's caching allocator that holds all
// of HBM), and latency-bound paths that cannot afford the device-wide
// synchronisation that cudaMalloc / cudaFree imply.  ahs_features_noalloc
// serves them: it runs the same three feature kernels as ahs_features, but its
// scratch lives in one file-scope device array of fixed size
// (kNoAllocScratchBytes) that every GPU holds from the moment the library's
// module is loaded there until the process exits.  It needs no ahs_ctx,
// allocates nothing, and the caller passes the input and receives the result
// on the host.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 48ull << 20;   // 48 MiB
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceSetup {
    bool done = false;
    ahs_status status = AHS_OK;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    int sms = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Once per device, with that device current: resolve the scratch address and
// check that this device's feature kernels fit in it.  Only a definite answer
// is kept (the address, or "this device has too many SMs"); a failed CUDA call
// is returned and retried by the next call.
ahs_status setup_device(int dev, DeviceSetup** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? AHS_ERR_OOM : AHS_ERR_CUDA;
        }
        if (a256(sizeof(ahs::DevFeatures)) + ahs::features_scratch_bytes(sms) >
            kNoAllocScratchBytes) {
            s.status = AHS_ERR_RANGE;   // more SMs than the fixed scratch was sized for
        } else {
            s.status = AHS_OK;
            s.base = static_cast<unsigned char*>(ptr);
            s.sms = sms;
        }
        s.done = true;
    }
    *out = &s;
    return s.status;
}

}  // namespace

extern "C" ahs_status ahs_features_noalloc(const void* d_keys, uint64_t n, ahs_key_type type,
                                           void* stream, ahs_features_t* h_out) {
    if (!h_out) return AHS_ERR_INVALID_ARG;
    if (type < AHS_U32 || type > AHS_I64) return AHS_ERR_DTYPE;
    if (n && !d_keys) return AHS_ERR_INVALID_ARG;
    if (n > AHS_NOALLOC_MAX_KEYS) return AHS_ERR_RANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AHS_ERR_CUDA;
    DeviceSetup* s = nullptr;
    ahs_status rc = setup_device(dev, &s);
    if (rc != AHS_OK) return rc;
    std::memset(h_out, 0, sizeof(*h_out));
    if (n == 0) return AHS_OK;

    // Carve the fixed scratch: the feature record first, then the kernels'
    // partials, per-CTA histogram slabs, exact histogram and entropy partials.
    unsigned char* p = s->base;
    ahs::FeatureScratch fs{};
    fs.rec = reinterpret_cast<ahs::DevFeatures*>(p);
    p += a256(sizeof(ahs::DevFeatures));
    fs.k1_partials = reinterpret_cast<unsigned long long*>(p);
    p += a256(3 * sizeof(unsigned long long) * 4 * (size_t)s->sms);
    fs.slabs = reinterpret_cast<uint32_t*>(p);
    p += a256((size_t)s->sms * ahs::kMaxBins * sizeof(uint32_t));
    fs.hist = reinterpret_cast<unsigned long long*>(p);
    p += a256(ahs::kMaxBins * sizeof(unsigned long long));
    fs.ent_partials = reinterpret_cast<double*>(p);

    const ahs::KeyDesc kd = ahs::key_desc(type);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The scratch keeps the previous call's contents: the record holds the
    // kernels' block counters, which must start at zero.
    cudaError_t e = cudaMemsetAsync(fs.rec, 0, sizeof(ahs::DevFeatures), st);
    if (e == cudaSuccess) e = ahs::launch_features(d_keys, n, kd, fs, s->sms, st);
    ahs::DevFeatures r;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&r, fs.rec, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // A packed histogram counter wrapped: count again in the exact layout.
    if (e == cudaSuccess && r.k2_wrapped) {
        e = ahs::launch_features_split_retry(d_keys, n, kd, fs, s->sms, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&r, fs.rec, sizeof(r), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? AHS_ERR_OOM : AHS_ERR_CUDA;
    h_out->n = r.n;
    h_out->min_bits = r.min_ord ^ kd.flip;
    h_out->max_bits = r.max_ord ^ kd.flip;
    h_out->span = r.span;
    h_out->hist_shift = r.shift;
    h_out->nbins = r.nbins;
    h_out->entropy_bits = r.entropy;
    h_out->entropy_norm = r.entropy_norm;
    h_out->descents = r.descents;
    h_out->ascents = r.ascents;
    return AHS_OK;
}
