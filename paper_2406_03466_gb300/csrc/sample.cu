// Shot sampling of one state (the bitstring counts a measurement of every
// qubit in the Z basis returns, Sec. 3 and Sec. 4.2): shot s takes the
// first basis index b whose cumulative probability exceeds u_s times the
// total, P(b) = |psi_b|^2 in FP64.  The uniforms u_s are inputs, so the
// draw is reproducible and checkable.  Three kernels: FP64 sums of P over
// chunks of 1024 amplitudes, an exclusive prefix over the chunks (one
// block), and one thread per shot (binary search over the chunk prefix,
// then a walk through the chunk), with optional histogram counts.
#include <cuda_runtime.h>

#include <cstdint>

#include "sample.h"

namespace svk {
namespace {

constexpr int kChunkBits = 10;
constexpr int kChunk = 1 << kChunkBits;

template <typename C> __device__ __forceinline__ double prob(const C a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// S[k] = sum of P over chunk k (one block of 256 threads per chunk).
template <typename C>
__global__ void k_chunk_sums(const C *psi, int64_t dim, double *S) {
    __shared__ double red[8];
    const int64_t k = blockIdx.x;
    double v = 0.0;
    for (int64_t j = k * kChunk + threadIdx.x; j < dim && j < (k + 1) * kChunk; j += blockDim.x)
        v += prob(psi[j]);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        S[k] = s;
    }
}

// In place: S[k] <- S[0] + ... + S[k - 1]; S[K] <- the total.  One block of
// 1024 threads: each thread sums a contiguous run, a block scan of the runs,
// then each run is rewritten.
__global__ void k_chunk_prefix(double *S, int64_t K) {
    __shared__ double run[1024];
    const int T = blockDim.x, tid = threadIdx.x;
    const int64_t per = (K + T - 1) / T, lo = per * tid, hi = lo + per < K ? lo + per : K;
    double s = 0.0;
    for (int64_t k = lo; k < hi; ++k) s += S[k];
    run[tid] = s;
    __syncthreads();
    if (tid == 0) {  // exclusive scan of the T run sums (T = 1024: cheap)
        double acc = 0.0;
        for (int i = 0; i < T; ++i) {
            const double x = run[i];
            run[i] = acc;
            acc += x;
        }
        S[K] = acc;
    }
    __syncthreads();
    double acc = run[tid];
    for (int64_t k = lo; k < hi; ++k) {
        const double x = S[k];
        S[k] = acc;
        acc += x;
    }
}

template <typename C>
__global__ void k_sample(const C *psi, int64_t dim, const double *S, int64_t K, const double *u,
                         int64_t n_shots, int64_t *samples, unsigned long long *counts) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_shots;
         s += (int64_t)gridDim.x * blockDim.x) {
        const double x = u[s] * S[K];
        // last chunk k with S[k] <= x
        int64_t lo = 0, hi = K - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (S[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        double acc = S[lo];
        const int64_t j0 = lo * kChunk, j1 = j0 + kChunk < dim ? j0 + kChunk : dim;
        int64_t b = j1 - 1;  // rounding at the very end falls on the chunk's last index
        for (int64_t j = j0; j < j1; ++j) {
            acc += prob(psi[j]);
            if (acc > x) {
                b = j;
                break;
            }
        }
        samples[s] = b;
        if (counts) atomicAdd(&counts[b], 1ull);
    }
}

}  // namespace

size_t sample_scratch_bytes(int n) {
    const int64_t K = ((int64_t(1) << n) + kChunk - 1) >> kChunkBits;
    return sizeof(double) * (size_t)(K + 1);
}

cudaError_t launch_sample(int c128, int n, const void *psi, const double *uniforms,
                          int64_t n_shots, int64_t *samples, int64_t *counts, double *scratch,
                          cudaStream_t st) {
    const int64_t dim = int64_t(1) << n, K = (dim + kChunk - 1) >> kChunkBits;
    if (counts) {
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)dim, st);
        if (e != cudaSuccess) return e;
    }
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(counts);
    const int gs = (int)((n_shots + 255) / 256 < 65536 ? (n_shots + 255) / 256 : 65536);
    if (c128) {
        k_chunk_sums<double2><<<(unsigned)K, 256, 0, st>>>((const double2 *)psi, dim, scratch);
        k_chunk_prefix<<<1, 1024, 0, st>>>(scratch, K);
        if (n_shots > 0)
            k_sample<double2><<<gs, 256, 0, st>>>((const double2 *)psi, dim, scratch, K, uniforms,
                                                  n_shots, samples, cnt);
    } else {
        k_chunk_sums<float2><<<(unsigned)K, 256, 0, st>>>((const float2 *)psi, dim, scratch);
        k_chunk_prefix<<<1, 1024, 0, st>>>(scratch, K);
        if (n_shots > 0)
            k_sample<float2><<<gs, 256, 0, st>>>((const float2 *)psi, dim, scratch, K, uniforms,
                                                 n_shots, samples, cnt);
    }
    return cudaGetLastError();
}

}  // namespace svk
