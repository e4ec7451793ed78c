// FP32 instantiation of the pass kernels, and the line-search bookkeeping kernel.
#define DFT_DEFINE_FINALIZE
#include "passes_impl.cuh"

template struct Passes<float>;

cudaError_t finalize_init_attributes() { return cudaSuccess; }

void launch_finalize(cudaStream_t st, Ctl* ctl, const double* red_sum, int nsum, const float* red_max, int nmax,
                     int op, double inv_count, double alpha_fixed, double n3_bound, double alpha_floor) {
    dftk::k_finalize<<<1, dftk::kThreads, 0, st>>>(ctl, red_sum, nsum, red_max, nmax, op, inv_count, alpha_fixed,
                                                  n3_bound, alpha_floor);
}
