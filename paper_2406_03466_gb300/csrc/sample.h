// Shot sampling of one state (sample.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace svk {

// FP64 scratch the sampler needs for a state of n qubits.
size_t sample_scratch_bytes(int n);
// samples[s] = the basis index of shot s drawn with uniforms[s] in [0, 1);
// counts (device [2^n], or null) = the histogram of the samples.
cudaError_t launch_sample(int c128, int n, const void *psi, const double *uniforms,
                          int64_t n_shots, int64_t *samples, int64_t *counts, double *scratch,
                          cudaStream_t st);

}  // namespace svk
