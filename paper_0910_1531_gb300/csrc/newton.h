// Elementwise and reduction kernels of the Newton-Krylov solver over an S N field (host
// launchers; newton.cu).  Excluded voxels (V = +inf) carry 0 in every Krylov vector.
#pragma once

#include <cuda_runtime.h>

template <typename Real>
class NkVec {
public:
    NkVec(cudaStream_t st, long long n, int grid);
    // F = log rho - log g (accessible voxels)
    cudaError_t residual(const Real* rho, const Real* g, const Real* V, Real* F) const;
    // out = rho exp(s d) (accessible voxels)
    cudaError_t step(const Real* rho, const Real* d, double s, const Real* V, Real* out) const;
    // out = (F(rho_p) - F) / eps from rho_p and its G
    cudaError_t jv(const Real* rho_p, const Real* g_p, const Real* F, const Real* V, double eps, Real* out) const;
    // y = alpha x + beta y
    cudaError_t axpby(double alpha, const Real* x, double beta, Real* y) const;
    // <a, b> in FP64 (synchronises the stream); partial_dev / partial_host hold `grid` doubles
    cudaError_t dot(const Real* a, const Real* b, double* partial_dev, double* partial_host, double* out) const;

private:
    cudaStream_t st_;
    long long n_;
    int grid_;
};
