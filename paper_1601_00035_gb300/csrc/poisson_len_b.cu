// Poisson FFT passes for the lengths of unit b (poisson_passes.hpp).
#include "poisson_kernels.cuh"

namespace lgf {

cudaError_t poisson_tw_upload_b() { return fft::upload_tw64(); }

#define INST(n) template struct PoissonPasses<n, float>; template struct PoissonPasses<n, double>;
LGF_POISSON_LENGTHS_B(INST)
#undef INST

}  // namespace lgf
