// The plain complex128 form used as the comparison point: one circuit at a
// time, one kernel launch per gate and one per Pauli term, the state in
// device memory.  Nothing here is batched, fused or staged on chip.
#include <cuda_runtime.h>

#include "kernels.h"

namespace svk {
namespace {

__global__ void k_plain_init(double2 *psi, int64_t dim, int64_t ref) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x)
        psi[j] = make_double2(j == ref ? 1.0 : 0.0, 0.0);
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One thread per index pair (j, j | 2^q) with bit q of j clear.
__global__ void k_plain_u1(double2 *psi, int n, int q, double2 m0, double2 m1, double2 m2,
                           double2 m3) {
    const int64_t pairs = int64_t(1) << (n - 1);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = p & ((int64_t(1) << q) - 1);
        const int64_t j0 = ((p >> q) << (q + 1)) | lo, j1 = j0 | (int64_t(1) << q);
        const double2 x = psi[j0], y = psi[j1];
        const double2 a = cm(m0, x), b = cm(m1, y), c = cm(m2, x), d = cm(m3, y);
        psi[j0] = make_double2(a.x + b.x, a.y + b.y);
        psi[j1] = make_double2(c.x + d.x, c.y + d.y);
    }
}

__global__ void k_plain_cx(double2 *psi, int n, int c, int t) {
    const int64_t pairs = int64_t(1) << (n - 1);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = p & ((int64_t(1) << t) - 1);
        const int64_t j0 = ((p >> t) << (t + 1)) | lo, j1 = j0 | (int64_t(1) << t);
        if ((j0 >> c) & 1) {
            const double2 x = psi[j0];
            psi[j0] = psi[j1];
            psi[j1] = x;
        }
    }
}

__global__ void k_plain_cz(double2 *psi, int n, int a, int b) {
    const int64_t dim = int64_t(1) << n;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x)
        if (((j >> a) & 1) && ((j >> b) & 1)) psi[j] = make_double2(-psi[j].x, -psi[j].y);
}

// acc += coeff * Re(i^phase sum_j (-1)^{|j & z|} conj(psi_{j^x}) psi_j)
__global__ void k_plain_term(const double2 *psi, int n, uint32_t x, uint32_t z, int phase,
                             double coeff, double *acc) {
    __shared__ double red[32];
    const int64_t dim = int64_t(1) << n;
    double sre = 0.0, sim = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = psi[j], q = psi[j ^ x];
        double wr = q.x * p.x + q.y * p.y, wi = q.x * p.y - q.y * p.x;
        if (__popcll((unsigned long long)(j & z)) & 1) {
            wr = -wr;
            wi = -wi;
        }
        sre += wr;
        sim += wi;
    }
    double v = phase == 0 ? sre : phase == 1 ? -sim : phase == 2 ? -sre : sim;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(acc, coeff * s);
    }
}

void grid_for(int64_t work, int *blocks, int *threads) {
    *threads = 256;
    int64_t b = (work + 255) / 256;
    if (b > 1184) b = 1184;
    if (b < 1) b = 1;
    *blocks = (int)b;
}

}  // namespace

cudaError_t launch_plain_init(double2 *psi, int n, int64_t ref, cudaStream_t st) {
    int b, t;
    grid_for(int64_t(1) << n, &b, &t);
    k_plain_init<<<b, t, 0, st>>>(psi, int64_t(1) << n, ref);
    return cudaGetLastError();
}

cudaError_t launch_plain_u1(double2 *psi, int n, int q, const double2 m[4], cudaStream_t st) {
    int b, t;
    grid_for(int64_t(1) << (n - 1), &b, &t);
    k_plain_u1<<<b, t, 0, st>>>(psi, n, q, m[0], m[1], m[2], m[3]);
    return cudaGetLastError();
}

cudaError_t launch_plain_cx(double2 *psi, int n, int c, int t_, cudaStream_t st) {
    int b, t;
    grid_for(int64_t(1) << (n - 1), &b, &t);
    k_plain_cx<<<b, t, 0, st>>>(psi, n, c, t_);
    return cudaGetLastError();
}

cudaError_t launch_plain_cz(double2 *psi, int n, int a, int bq, cudaStream_t st) {
    int b, t;
    grid_for(int64_t(1) << n, &b, &t);
    k_plain_cz<<<b, t, 0, st>>>(psi, n, a, bq);
    return cudaGetLastError();
}

cudaError_t launch_plain_term(const double2 *psi, int n, uint32_t x, uint32_t z, int phase,
                              double coeff, double *acc, cudaStream_t st) {
    int b, t;
    grid_for(int64_t(1) << n, &b, &t);
    k_plain_term<<<b, t, 0, st>>>(psi, n, x, z, phase, coeff, acc);
    return cudaGetLastError();
}

}  // namespace svk
