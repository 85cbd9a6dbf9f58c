// Per-launch tracing: when a context has tracing on, every kernel launch of a
// call is bracketed by two CUDA events recorded on the launching stream, so
// the device duration of each kernel can be read back afterwards.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <vector>

namespace ahs {

// AHS_DEBUG_SYNC=1 in the environment: synchronise after every traced launch
// and name the kernel whose execution failed (debugging aid).
inline bool debug_sync() {
    static const bool on = [] {
        const char* v = std::getenv("AHS_DEBUG_SYNC");
        return v && v[0] == '1';
    }();
    return on;
}

struct TraceRecord {
    const char* name;
    uint64_t items;       // keys the launch processes (0 if not meaningful)
    cudaEvent_t a, b;
};

struct Tracer {
    bool on = false;
    std::vector<TraceRecord> records;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

// The tracer of the context whose call is running on this thread (or null).
extern thread_local Tracer* g_tracer;

class TraceScope {
public:
    TraceScope(const char* name, uint64_t items, cudaStream_t st) : st_(st), name_(name) {
        if (g_tracer && g_tracer->on) {
            rec_.name = name;
            rec_.items = items;
            rec_.a = g_tracer->take();
            rec_.b = g_tracer->take();
            cudaEventRecord(rec_.a, st);
            active_ = true;
        }
    }
    ~TraceScope() {
        if (debug_sync()) {
            cudaError_t e = cudaStreamSynchronize(st_);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) std::fprintf(stderr, "[ahs] kernel %s failed: %s\n", name_, cudaGetErrorString(e));
        }
        if (active_) {
            cudaEventRecord(rec_.b, st_);
            g_tracer->records.push_back(rec_);
        }
    }
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;

private:
    cudaStream_t st_;
    const char* name_;
    TraceRecord rec_{};
    bool active_ = false;
};

// Installs a context's tracer for the duration of one API call.
class TracerGuard {
public:
    explicit TracerGuard(Tracer* t) : saved_(g_tracer) { g_tracer = t; }
    ~TracerGuard() { g_tracer = saved_; }

private:
    Tracer* saved_;
};

}  // namespace ahs
