// One (precision, axis length) instantiation of the pass kernels.  Compiled once per pair
// with -DDFT_INST_REAL=<float|double> -DDFT_INST_N=<0|32|48|64|96|128|256>.
#include "launch_impl.cuh"

#ifndef DFT_INST_REAL
#error "DFT_INST_REAL must be defined"
#endif
#ifndef DFT_INST_N
#error "DFT_INST_N must be defined"
#endif

template struct LaunchX<DFT_INST_REAL, DFT_INST_N>;
template struct LaunchY<DFT_INST_REAL, DFT_INST_N>;
template struct LaunchZ<DFT_INST_REAL, DFT_INST_N>;
