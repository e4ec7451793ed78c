// FP64 instantiation of the pass kernels (the all-FP64 method).
#include "passes_impl.cuh"

template struct Passes<double>;
