// Seeded synthetic workloads, device side: the same counter-based definitions
// as gen/host.py, bit for bit (SplitMix64 output function on a counter,
// Lemire multiply-shift for bounded integers).  Inputs only: nothing here is
// part of the sorting method.  Built as gen/libahsgen.so, separate from the
// sorting library.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ unsigned long long stream_key(unsigned long long seed,
                                                                  unsigned long long stream) {
    return mix64(seed * kGolden + mix64(stream + kGolden));
}

__device__ __forceinline__ unsigned long long draw(unsigned long long key, unsigned long long i) {
    return mix64(key + (i + 1) * kGolden);
}

__global__ void k_uniform_u32(uint32_t* out, unsigned long long n, unsigned long long key,
                              unsigned long long m, unsigned long long start) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride)
        out[i] = (uint32_t)(((draw(key, start + i) >> 32) * m) >> 32);
}

__global__ void k_zipf_u32(uint32_t* out, unsigned long long n, unsigned long long key,
                           const double* cdf, const uint32_t* values, uint32_t nv,
                           unsigned long long start) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const double u = (double)(draw(key, start + i) >> 11) * 0x1.0p-53;
        // first index with cdf[idx] > u
        uint32_t lo = 0, hi = nv;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cdf[mid] > u) hi = mid;
            else lo = mid + 1;
        }
        out[i] = values[lo < nv ? lo : nv - 1];
    }
}

__global__ void k_ramp_steps(unsigned long long* out, unsigned long long n, unsigned long long key,
                             unsigned long long m) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride)
        out[i] = i == 0 ? 0ull : __umul64hi(draw(key, i), m);
}

__global__ void k_ramp_replace(unsigned long long* t, unsigned long long n, unsigned long long key_p,
                               unsigned long long key_v, unsigned long long thresh53,
                               unsigned long long t0, unsigned long long range) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        if ((draw(key_p, i) >> 11) < thresh53) {
            const unsigned long long r = draw(key_v, i);
            t[i] = t0 + (range == 0 ? r : __umul64hi(r, range));
        }
    }
}

// Sequential swaps of (i, j) pairs: one thread keeps the sequential semantics.
__global__ void k_swaps_u32(uint32_t* a, unsigned long long n, unsigned long long swaps,
                            unsigned long long key) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (unsigned long long t = 0; t < swaps; ++t) {
        const unsigned long long i = __umul64hi(draw(key, 2 * t), n);
        const unsigned long long j = __umul64hi(draw(key, 2 * t + 1), n);
        const uint32_t x = a[i];
        a[i] = a[j];
        a[j] = x;
    }
}

// Second workload family: Gaussian-shaped int32 keys by an integer
// Irwin-Hall sum (12 uniform 32-bit integers from 6 draws per key), and
// 60-bit k-mer keys of a synthetic repetitive genome (as gen/host.py).
__global__ void k_gaussian_i32(int32_t* out, unsigned long long n, unsigned long long key,
                               long long sigma_q16, unsigned long long start) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        long long S = 0;
        for (int m = 0; m < 6; ++m) {
            const unsigned long long r = draw(key, 6 * (start + i) + m);
            S += (long long)(r >> 32) + (long long)(r & 0xffffffffull);
        }
        const long long d = S - 6ll * 4294967295ll;
        out[i] = (int32_t)((d * sigma_q16) >> 48);
    }
}

constexpr unsigned long long kKmerBlock = 1000, kKmerRepeats = 16, kKmerLen = 30;
constexpr unsigned long long kKmerMut53 = 90071992547410ull;

__device__ __forceinline__ unsigned long long kmer_base(unsigned long long p, unsigned long long key_rep,
                                                        unsigned long long key_unit,
                                                        unsigned long long key_mut) {
    const unsigned long long r = __umul64hi(draw(key_rep, p / kKmerBlock), kKmerRepeats);
    const unsigned long long u = draw(key_unit, r * kKmerBlock + p % kKmerBlock) >> 62;
    const unsigned long long m = draw(key_mut, p);
    return (m >> 11) < kKmerMut53 ? (m & 3ull) : u;
}

__global__ void k_kmer_u64(unsigned long long* out, unsigned long long n, unsigned long long key_rep,
                           unsigned long long key_unit, unsigned long long key_mut,
                           unsigned long long start) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        unsigned long long k = 0;
        for (unsigned long long j = 0; j < kKmerLen; ++j)
            k |= kmer_base(start + i + j, key_rep, key_unit, key_mut) << (2 * (kKmerLen - 1 - j));
        out[i] = k;
    }
}

__global__ void k_replace_u32(uint32_t* a, unsigned long long n, unsigned long long key_p,
                              unsigned long long key_v, unsigned long long thresh53) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride)
        if ((draw(key_p, i) >> 11) < thresh53) a[i] = (uint32_t)(draw(key_v, i) >> 32);
}

__host__ __device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

// Batch of segments (one CTA each): type 0 uniform below 4096, 1 Zipf over
// 1,024 distinct values of the segment, 2 and 3 uniform 32-bit (type 3 is
// sorted and swapped afterwards).  Streams per segment s: keys 16 + 4 s,
// Zipf values 16 + 4 s + 1 (as gen/host.py segment_stream).
__global__ void k_batch_u32(uint32_t* out, const unsigned long long* offs, const unsigned char* types,
                            unsigned long long seed, const double* cdf, uint32_t nv) {
    const unsigned s = blockIdx.x;
    const unsigned long long b = offs[s], n = offs[s + 1] - offs[s];
    const unsigned long long key = stream_key(seed, 16ull + 4ull * s);
    const unsigned t = types[s];
    uint32_t k1 = 0, k2 = 0;
    if (t == 1) {
        const unsigned long long kz = mix64(stream_key(seed, 16ull + 4ull * s + 1) + kGolden);
        k1 = (uint32_t)kz;
        k2 = (uint32_t)(kz >> 32);
    }
    for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long r = draw(key, i);
        uint32_t v;
        if (t == 0) {
            v = (uint32_t)(((r >> 32) * 4096ull) >> 32);
        } else if (t == 1) {
            const double u = (double)(r >> 11) * 0x1.0p-53;
            uint32_t lo = 0, hi = nv;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (cdf[mid] > u) hi = mid;
                else lo = mid + 1;
            }
            const uint32_t rank = lo < nv ? lo : nv - 1;
            v = hash32(rank ^ k1) ^ k2;
        } else {
            v = (uint32_t)(r >> 32);
        }
        out[b + i] = v;
    }
}

// Per listed segment, its floor(n / 100) sequential swaps (one thread each).
__global__ void k_batch_swaps(uint32_t* out, const unsigned long long* offs, const unsigned* segs,
                              unsigned nlist, unsigned long long seed) {
    const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nlist) return;
    const unsigned s = segs[j];
    const unsigned long long b = offs[s], n = offs[s + 1] - offs[s];
    const unsigned long long key = stream_key(seed, 16ull + 4ull * s + 2);
    uint32_t* a = out + b;
    for (unsigned long long t = 0; t < n / 100; ++t) {
        const unsigned long long i = __umul64hi(draw(key, 2 * t), n);
        const unsigned long long k = __umul64hi(draw(key, 2 * t + 1), n);
        const uint32_t x = a[i];
        a[i] = a[k];
        a[k] = x;
    }
}

unsigned grid(unsigned long long n) {
    unsigned long long g = (n + 255) / 256;
    return (unsigned)(g < 8192 ? (g ? g : 1) : 8192);
}

}  // namespace

extern "C" {

int gen_uniform_u32(void* out, unsigned long long n, unsigned long long seed,
                    unsigned long long stream, unsigned long long m, unsigned long long start,
                    void* st) {
    if (n == 0) return 0;
    k_uniform_u32<<<grid(n), 256, 0, (cudaStream_t)st>>>((uint32_t*)out, n, stream_key(seed, stream),
                                                         m, start);
    return (int)cudaGetLastError();
}

int gen_zipf_u32(void* out, unsigned long long n, unsigned long long seed, unsigned long long stream,
                 const void* d_cdf, const void* d_values, unsigned nv, unsigned long long start,
                 void* st) {
    if (n == 0) return 0;
    k_zipf_u32<<<grid(n), 256, 0, (cudaStream_t)st>>>((uint32_t*)out, n, stream_key(seed, stream),
                                                      (const double*)d_cdf, (const uint32_t*)d_values,
                                                      nv, start);
    return (int)cudaGetLastError();
}

int gen_ramp_steps(void* out, unsigned long long n, unsigned long long seed, unsigned long long m,
                   void* st) {
    if (n == 0) return 0;
    k_ramp_steps<<<grid(n), 256, 0, (cudaStream_t)st>>>((unsigned long long*)out, n,
                                                        stream_key(seed, 1), m);
    return (int)cudaGetLastError();
}

int gen_ramp_replace(void* t, unsigned long long n, unsigned long long seed,
                     unsigned long long thresh53, unsigned long long t0, unsigned long long range,
                     void* st) {
    if (n == 0) return 0;
    k_ramp_replace<<<grid(n), 256, 0, (cudaStream_t)st>>>((unsigned long long*)t, n,
                                                          stream_key(seed, 2), stream_key(seed, 3),
                                                          thresh53, t0, range);
    return (int)cudaGetLastError();
}

int gen_swaps_u32(void* a, unsigned long long n, unsigned long long swaps, unsigned long long seed,
                  unsigned long long stream, void* st) {
    if (n == 0 || swaps == 0) return 0;
    k_swaps_u32<<<1, 1, 0, (cudaStream_t)st>>>((uint32_t*)a, n, swaps, stream_key(seed, stream));
    return (int)cudaGetLastError();
}

int gen_gaussian_i32(void* out, unsigned long long n, unsigned long long seed,
                     unsigned long long stream, long long sigma_q16, unsigned long long start,
                     void* st) {
    if (n == 0) return 0;
    k_gaussian_i32<<<grid(n), 256, 0, (cudaStream_t)st>>>((int32_t*)out, n, stream_key(seed, stream),
                                                          sigma_q16, start);
    return (int)cudaGetLastError();
}

int gen_kmer_u64(void* out, unsigned long long n, unsigned long long seed, unsigned long long stream,
                 unsigned long long start, void* st) {
    if (n == 0) return 0;
    k_kmer_u64<<<grid(n), 256, 0, (cudaStream_t)st>>>((unsigned long long*)out, n,
                                                      stream_key(seed, stream),
                                                      stream_key(seed, stream + 1),
                                                      stream_key(seed, stream + 2), start);
    return (int)cudaGetLastError();
}

int gen_replace_u32(void* a, unsigned long long n, unsigned long long seed, unsigned long long stream,
                    unsigned long long thresh53, void* st) {
    if (n == 0) return 0;
    k_replace_u32<<<grid(n), 256, 0, (cudaStream_t)st>>>((uint32_t*)a, n, stream_key(seed, stream),
                                                         stream_key(seed, stream + 1), thresh53);
    return (int)cudaGetLastError();
}

// Host-side tables of the Zipf workloads (as gen/host.py zipf_cdf and
// zipf_values): the fp64 CDF of p_r ~ r^-s by sequential summation in rank
// order (last entry 1.0), and the distinct values hash32(r ^ k1) ^ k2.
void gen_zipf_cdf_host(double* out, unsigned nv, double s) {
    double total = 0.0;
    for (unsigned r = 1; r <= nv; ++r) total += pow((double)r, -s);
    double acc = 0.0;
    for (unsigned r = 1; r <= nv; ++r) {
        acc += pow((double)r, -s);
        out[r - 1] = acc / total;
    }
    if (nv) out[nv - 1] = 1.0;
}

void gen_zipf_values_host(uint32_t* out, unsigned long long seed, unsigned long long stream,
                          unsigned nv) {
    const unsigned long long k = mix64(stream_key(seed, stream) + kGolden);   // draw 0
    const uint32_t k1 = (uint32_t)(k & 0xffffffffull), k2 = (uint32_t)(k >> 32);
    for (unsigned r = 0; r < nv; ++r) out[r] = hash32(r ^ k1) ^ k2;
}

int gen_batch_u32(void* out, const void* d_offs, const void* d_types, unsigned nseg,
                  unsigned long long seed, const void* d_cdf, unsigned nv, void* st) {
    if (nseg == 0) return 0;
    k_batch_u32<<<nseg, 256, 0, (cudaStream_t)st>>>((uint32_t*)out, (const unsigned long long*)d_offs,
                                                    (const unsigned char*)d_types, seed,
                                                    (const double*)d_cdf, nv);
    return (int)cudaGetLastError();
}

int gen_batch_swaps(void* out, const void* d_offs, const void* d_segs, unsigned nlist,
                    unsigned long long seed, void* st) {
    if (nlist == 0) return 0;
    k_batch_swaps<<<(nlist + 127) / 128, 128, 0, (cudaStream_t)st>>>(
        (uint32_t*)out, (const unsigned long long*)d_offs, (const unsigned*)d_segs, nlist, seed);
    return (int)cudaGetLastError();
}

}  // extern "C"
