// Poisson FFT passes for the lengths of unit a (poisson_passes.hpp).
#include "poisson_kernels.cuh"

namespace lgf {

cudaError_t poisson_tw_upload_a() { return fft::upload_tw64(); }

#define INST(n) template struct PoissonPasses<n, float>; template struct PoissonPasses<n, double>;
LGF_POISSON_LENGTHS_A(INST)
#undef INST

}  // namespace lgf
