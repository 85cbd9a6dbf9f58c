// Host buffers in, host buffers out: a sequence of arrays in host memory, each
// sorted by ahs_sort, with the copy of array i + 1 to the device and of array
// i - 1 back to the host running while array i is sorted.  The context keeps
// the three streams (copy in, sort, copy out), the per-buffer events and two
// device buffer pairs between calls, so consecutive calls overlap as well:
// a call's first copy in waits only for the buffer pair it reuses.
#include <cstring>
#include <new>

#include "ctx.h"
#include "internal.h"

namespace ahs {

struct HostPipe {
    cudaStream_t in = nullptr, sort = nullptr, out = nullptr;
    cudaEvent_t loaded[2] = {}, consumed[2] = {}, freed[2] = {}, entry = nullptr;
    void* keys[2] = {};     // device input of each pair
    void* res[2] = {};      // device output of each pair
    uint32_t* vin[2] = {};  // payload, when the arrays carry one
    uint32_t* vres[2] = {};
    size_t key_cap = 0, val_cap = 0;   // bytes of each buffer
    uint32_t turn = 0;                 // pair the next array uses

    cudaError_t init() {
        if (in) return cudaSuccess;
        cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sort, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&loaded[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&consumed[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&entry, cudaEventDisableTiming);
        return e;
    }
    void drain() {
        if (in) cudaStreamSynchronize(in);
        if (sort) cudaStreamSynchronize(sort);
        if (out) cudaStreamSynchronize(out);
    }
    // Buffers of at least kb key bytes and vb payload bytes (waits for the
    // streams before replacing buffers that earlier calls may still use).
    cudaError_t reserve(size_t kb, size_t vb) {
        if (kb <= key_cap && vb <= val_cap) return cudaSuccess;
        drain();
        release_buffers();
        const size_t k2 = kb + kb / 8, v2 = vb ? vb + vb / 8 : 0;
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaMalloc(&keys[b], k2);
            if (e == cudaSuccess) e = cudaMalloc(&res[b], k2);
            if (e == cudaSuccess && v2) e = cudaMalloc(reinterpret_cast<void**>(&vin[b]), v2);
            if (e == cudaSuccess && v2) e = cudaMalloc(reinterpret_cast<void**>(&vres[b]), v2);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            release_buffers();
            return e;
        }
        key_cap = k2;
        val_cap = v2;
        return cudaSuccess;
    }
    void release_buffers() {
        for (int b = 0; b < 2; ++b) {
            if (keys[b]) cudaFree(keys[b]);
            if (res[b]) cudaFree(res[b]);
            if (vin[b]) cudaFree(vin[b]);
            if (vres[b]) cudaFree(vres[b]);
            keys[b] = res[b] = nullptr;
            vin[b] = vres[b] = nullptr;
        }
        key_cap = val_cap = 0;
    }
    ~HostPipe() {
        drain();
        release_buffers();
        for (int b = 0; b < 2; ++b) {
            if (loaded[b]) cudaEventDestroy(loaded[b]);
            if (consumed[b]) cudaEventDestroy(consumed[b]);
            if (freed[b]) cudaEventDestroy(freed[b]);
        }
        if (entry) cudaEventDestroy(entry);
        if (in) cudaStreamDestroy(in);
        if (sort) cudaStreamDestroy(sort);
        if (out) cudaStreamDestroy(out);
    }
};

void destroy_host_pipe(HostPipe* p) { delete p; }

}  // namespace ahs

using namespace ahs;

extern "C" ahs_status ahs_sort_host(ahs_ctx* ctx, const ahs_host_array_t* arrays, uint32_t count,
                                    ahs_key_type type, ahs_strategy force, void* stream,
                                    int32_t wait, ahs_strategy* strategies) {
    if (!ctx || ctx->device < 0 || (count && !arrays)) return AHS_ERR_INVALID_ARG;
    if (type < AHS_U32 || type > AHS_I64) return AHS_ERR_DTYPE;
    if (force < AHS_AUTO || force > AHS_GENERAL) return AHS_ERR_INVALID_ARG;
    if (count == 0) return AHS_OK;
    const KeyDesc kd = key_desc(type);
    const bool pay = arrays[0].h_vals_in != nullptr;
    uint64_t cap = 0;
    for (uint32_t i = 0; i < count; ++i) {
        const ahs_host_array_t& a = arrays[i];
        if (a.n && (!a.h_keys_in || !a.h_keys_out)) return AHS_ERR_INVALID_ARG;
        if ((a.h_vals_in != nullptr) != pay || (pay && a.n && !a.h_vals_out)) return AHS_ERR_INVALID_ARG;
        cap = a.n > cap ? a.n : cap;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    if (!ctx->host_pipe) {
        ctx->host_pipe = new (std::nothrow) HostPipe();
        if (!ctx->host_pipe) return AHS_ERR_OOM;
    }
    HostPipe& P = *ctx->host_pipe;
    e = P.init();
    if (e == cudaSuccess) e = P.reserve(cap * kd.bytes, pay ? cap * 4 : 0);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    // The caller's earlier work (which may produce the host inputs) comes first.
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    e = cudaEventRecord(P.entry, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.in, P.entry, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.sort, P.entry, 0);
    if (e != cudaSuccess) return cuda_status(ctx, e);

    const uint32_t first = P.turn;
    auto load = [&](uint32_t i) -> cudaError_t {
        const uint32_t b = (first + i) % 2;
        const ahs_host_array_t& a = arrays[i];
        cudaError_t r = cudaStreamWaitEvent(P.in, P.consumed[b], 0);   // the last sort of pair b
        if (r == cudaSuccess && a.n)
            r = cudaMemcpyAsync(P.keys[b], a.h_keys_in, a.n * kd.bytes, cudaMemcpyHostToDevice, P.in);
        if (r == cudaSuccess && pay && a.n)
            r = cudaMemcpyAsync(P.vin[b], a.h_vals_in, a.n * 4, cudaMemcpyHostToDevice, P.in);
        if (r == cudaSuccess) r = cudaEventRecord(P.loaded[b], P.in);
        return r;
    };
    e = load(0);
    ahs_status rc = AHS_OK;
    for (uint32_t i = 0; i < count && e == cudaSuccess && rc == AHS_OK; ++i) {
        const uint32_t b = (first + i) % 2;
        const ahs_host_array_t& a = arrays[i];
        if (i + 1 < count) e = load(i + 1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P.sort, P.loaded[b], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P.sort, P.freed[b], 0);   // last copy out of b
        if (e != cudaSuccess) break;
        ahs_sort_info_t info{};
        rc = ahs_sort(ctx, P.keys[b], P.res[b], pay ? P.vin[b] : nullptr, pay ? P.vres[b] : nullptr,
                      a.n, type, force, P.sort, &info);
        if (rc != AHS_OK) break;
        if (strategies) strategies[i] = info.strategy;
        e = cudaEventRecord(P.consumed[b], P.sort);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P.out, P.consumed[b], 0);
        if (e == cudaSuccess && a.n)
            e = cudaMemcpyAsync(a.h_keys_out, P.res[b], a.n * kd.bytes, cudaMemcpyDeviceToHost, P.out);
        if (e == cudaSuccess && pay && a.n)
            e = cudaMemcpyAsync(a.h_vals_out, P.vres[b], a.n * 4, cudaMemcpyDeviceToHost, P.out);
        if (e == cudaSuccess) e = cudaEventRecord(P.freed[b], P.out);
    }
    P.turn = (first + count) % 2;
    if (rc != AHS_OK) return rc;
    if (e != cudaSuccess) return cuda_status(ctx, e);
    if (wait) {
        e = cudaStreamSynchronize(P.out);
        if (e == cudaSuccess) e = cudaStreamSynchronize(P.in);
        return cuda_status(ctx, e);
    }
    return AHS_OK;
}

extern "C" ahs_status ahs_wait_host(ahs_ctx* ctx, void* stream) {
    if (!ctx || ctx->device < 0) return AHS_ERR_INVALID_ARG;
    if (!ctx->host_pipe || !ctx->host_pipe->in) return AHS_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    HostPipe& P = *ctx->host_pipe;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    // Record the pipe's current tails and make the caller's stream wait for them.
    for (cudaStream_t s : {P.in, P.sort, P.out}) {
        cudaEvent_t ev = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, ev, 0);
        if (ev) cudaEventDestroy(ev);   // released once the wait has been enqueued
    }
    return cuda_status(ctx, e);
}
