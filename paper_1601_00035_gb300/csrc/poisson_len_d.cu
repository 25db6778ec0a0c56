// Poisson FFT passes for the lengths of unit d (poisson_passes.hpp).
#include "poisson_kernels.cuh"

namespace lgf {

cudaError_t poisson_tw_upload_d() { return fft::upload_tw64(); }

#define INST(n) template struct PoissonPasses<n, float>;
LGF_POISSON_LENGTHS_D(INST)
#undef INST

}  // namespace lgf
