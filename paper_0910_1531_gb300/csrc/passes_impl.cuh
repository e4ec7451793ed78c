// Definitions of the Passes<Real> launchers (included once per precision).
#pragma once

#include "kernels.cuh"
#include "passes.h"

namespace {
// Allow each kernel the device's opt-in shared memory per block minus its static shared memory.
template <typename K> cudaError_t set_max_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
}  // namespace

template <typename Real>
cudaError_t Passes<Real>::init_attributes() {
    cudaError_t e = cudaSuccess;
    cudaError_t r;
    if ((r = set_max_smem(dftk::k_xfwd<Real>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_yfft<Real, false>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_yfft<Real, true>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_zconv_fwd<Real>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xphi<Real>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_zconv_bwd<Real>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xupdate<Real>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xinv<Real>)) != cudaSuccess) e = r;
    return e;
}

template <typename Real>
void Passes<Real>::xfwd(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int ncomp, int lx, const Real* in,
                        C* out, const C* tw) {
    const long long rows = (long long)ncomp * g.ny * g.nz;
    const long long pairs = (rows + 1) / 2;
    const unsigned blocks = (unsigned)ceil_div(pairs, lx);
    dftk::k_xfwd<Real><<<blocks, dftk::kThreads, smem_x(g.nx, lx), st>>>(g, px, ncomp, lx, in, out, tw);
}

template <typename Real>
void Passes<Real>::yfft(cudaStream_t st, bool inv, const GridDesc& g, const AxisPlan& py, int T, int ncomp,
                        C* data, const C* tw) {
    dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.nz, (unsigned)ncomp);
    const size_t sm = smem_col(g.ny, T, 2);
    if (inv) dftk::k_yfft<Real, true><<<grid, dftk::kThreads, sm, st>>>(g, py, T, data, tw);
    else dftk::k_yfft<Real, false><<<grid, dftk::kThreads, sm, st>>>(g, py, T, data, tw);
}

template <typename Real>
void Passes<Real>::zconv_fwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                             int T, Real kfx, Real kfy, Real kfz, int want_psi, const C* in, C* slot_n,
                             C* slot_es, const C* tw) {
    dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.ny);
    dftk::k_zconv_fwd<Real><<<grid, dftk::kThreads, smem_col(g.nz, T, 7), st>>>(g, pz, sp, T, kfx, kfy, kfz,
                                                                                want_psi, in, slot_n, slot_es, tw);
}

template <typename Real>
void Passes<Real>::xphi(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl, const C* A,
                        const C* B, C* mat, C* phi, float* red_max, int* status, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    dftk::k_xphi<Real><<<blocks, dftk::kThreads, smem_x(g.nx, 5 * LR), st>>>(g, px, LR, ctl, A, B, mat, phi,
                                                                             red_max, status, tw);
}

template <typename Real>
void Passes<Real>::zconv_bwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                             int T, Real kfx, Real kfy, Real kfz, int flags, int ncomp_out, const Ctl* ctl, C* phi,
                             const C* esA, const C* esB, C* es_mat, const C* tw) {
    dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.ny);
    dftk::k_zconv_bwd<Real><<<grid, dftk::kThreads, smem_col(g.nz, T, 7), st>>>(
        g, pz, sp, T, kfx, kfy, kfz, flags, ncomp_out, ctl, phi, esA, esB, es_mat, tw);
}

template <typename Real>
void Passes<Real>::xupdate(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                           int LR, const Ctl* ctl, const C* cspec, const Real* rho0, const Real* rho1, const Real* V,
                           Real* rho_out, Real* g_out, double* red_sum, int* status, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    const int lpr = (sp.S + 1) / 2;
    dftk::k_xupdate<Real><<<blocks, dftk::kThreads, smem_x(g.nx, lpr * LR), st>>>(
        g, px, sp, LR, ctl, cspec, rho0, rho1, V, rho_out, g_out, red_sum, status, tw);
}

template <typename Real>
void Passes<Real>::xinv(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, int ncomp, const C* spec,
                        Real* out, Real* out_last, const Offsets<Real>& off, int cmax, float* red_max, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    const int lpr = (ncomp + 1) / 2;
    dftk::k_xinv<Real><<<blocks, dftk::kThreads, smem_x(g.nx, lpr * LR), st>>>(g, px, LR, ncomp, spec, out,
                                                                               out_last, off, cmax, red_max, tw);
}
