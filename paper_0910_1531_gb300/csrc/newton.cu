// Newton-Krylov solver of the fixed point rho = G(rho) (Sec. "Nonlinear solver" mentions
// Newton-GMRES as the alternative it tried): F(u) = u - log G(e^u) on the accessible voxels
// (u = log rho), Jacobian-vector products by finite differences of F (each one G evaluation),
// restarted GMRES with modified Gram-Schmidt and Givens rotations on the host, and a
// backtracking line search on |F|.  Elementwise kernels over the S N field here; G comes from
// the plan's Picard map.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "newton.h"

namespace {

constexpr int kNkThreads = 256;

template <typename Real>
__global__ void k_nk_residual(const Real* __restrict__ rho, const Real* __restrict__ g, const Real* __restrict__ V,
                              Real* __restrict__ F, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Real v = V[i];
        F[i] = (isinf(v) && v > Real(0)) ? Real(0) : log(rho[i]) - log(g[i]);
    }
}

// out = rho exp(s d) on accessible voxels, 0 elsewhere
template <typename Real>
__global__ void k_nk_step(const Real* __restrict__ rho, const Real* __restrict__ d, Real s, const Real* __restrict__ V,
                          Real* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Real v = V[i];
        out[i] = (isinf(v) && v > Real(0)) ? Real(0) : rho[i] * exp(s * d[i]);
    }
}

// out = ((log rho_p - log g_p) - F) / eps on accessible voxels
template <typename Real>
__global__ void k_nk_jv(const Real* __restrict__ rho_p, const Real* __restrict__ g_p, const Real* __restrict__ F,
                        const Real* __restrict__ V, Real inv_eps, Real* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Real v = V[i];
        out[i] = (isinf(v) && v > Real(0)) ? Real(0) : ((log(rho_p[i]) - log(g_p[i])) - F[i]) * inv_eps;
    }
}

// per-block partial sums of a * b, accumulated in FP64
template <typename Real>
__global__ void __launch_bounds__(kNkThreads) k_nk_dot(const Real* __restrict__ a, const Real* __restrict__ b,
                                                       long long n, double* __restrict__ partial) {
    __shared__ double sh[kNkThreads / 32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += double(a[i]) * double(b[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNkThreads / 32; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

// y = alpha x + beta y
template <typename Real>
__global__ void k_nk_axpby(Real alpha, const Real* __restrict__ x, Real beta, Real* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

}  // namespace

template <typename Real>
NkVec<Real>::NkVec(cudaStream_t st, long long n, int grid) : st_(st), n_(n), grid_(grid) {}

template <typename Real>
cudaError_t NkVec<Real>::residual(const Real* rho, const Real* g, const Real* V, Real* F) const {
    k_nk_residual<Real><<<grid_, kNkThreads, 0, st_>>>(rho, g, V, F, n_);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t NkVec<Real>::step(const Real* rho, const Real* d, double s, const Real* V, Real* out) const {
    k_nk_step<Real><<<grid_, kNkThreads, 0, st_>>>(rho, d, Real(s), V, out, n_);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t NkVec<Real>::jv(const Real* rho_p, const Real* g_p, const Real* F, const Real* V, double eps, Real* out) const {
    k_nk_jv<Real><<<grid_, kNkThreads, 0, st_>>>(rho_p, g_p, F, V, Real(1.0 / eps), out, n_);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t NkVec<Real>::axpby(double alpha, const Real* x, double beta, Real* y) const {
    k_nk_axpby<Real><<<grid_, kNkThreads, 0, st_>>>(Real(alpha), x, Real(beta), y, n_);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t NkVec<Real>::dot(const Real* a, const Real* b, double* partial_dev, double* partial_host, double* out) const {
    k_nk_dot<Real><<<grid_, kNkThreads, 0, st_>>>(a, b, n_, partial_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(partial_host, partial_dev, sizeof(double) * grid_, cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) return e;
    double t = 0.0;
    for (int i = 0; i < grid_; ++i) t += partial_host[i];
    *out = t;
    return cudaSuccess;
}

template class NkVec<float>;
template class NkVec<double>;
