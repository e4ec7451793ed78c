// Definitions of LaunchX / LaunchY / LaunchZ<Real, N> (included by kinst.cu once per pair).
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

// x pass: twiddles (nx) + two buffers of `lines` rows at the kernel's row pitch
template <typename C, int N> size_t smem_x_of(int nx, int lines) {
    const int pitch = N > 0 ? ct_row_pitch(N) : nx + 1;
    return (size_t(nx) + 2 * size_t(lines) * pitch) * sizeof(C) + 16;
}
template <typename C> size_t smem_col_of(int n, int T, int nbuf) { return (size_t(n) + size_t(nbuf) * T * n) * sizeof(C) + 16; }
}  // namespace

// ---------------------------------------------------------------------------------- x
template <typename Real, int N>
cudaError_t LaunchX<Real, N>::init() {
    cudaError_t e = cudaSuccess, r;
    if ((r = set_max_smem(dftk::k_xfwd<Real, N>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xphi<Real, N, 1>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xphi<Real, N, 2>)) != cudaSuccess) e = r;
    if constexpr (N > 0) {
        if ((r = set_max_smem(dftk::k_xphi_tma<Real, N, 1>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_xphi_tma<Real, N, 2>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_xphi_cpa<Real, N, 1>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_xphi_cpa<Real, N, 2>)) != cudaSuccess) e = r;
    }
    if ((r = set_max_smem(dftk::k_xupdate<Real, N, 1>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xupdate<Real, N, 2>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xcanon<Real, N>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xinv<Real, N>)) != cudaSuccess) e = r;
    if ((r = set_max_smem(dftk::k_xgrad<Real, N>)) != cudaSuccess) e = r;
    return e;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xfwd(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int ncomp, int lx,
                            const Real* in, C* out, const C* tw) {
    const long long rows = (long long)ncomp * g.ny * g.nz;
    const unsigned blocks = (unsigned)ceil_div((rows + 1) / 2, lx);
    launch_k(dftk::k_xfwd<Real, N>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, lx), st, g.pdl, g, px, ncomp, lx, in, out, tw);
    return cudaSuccess;
}

namespace {
// The persistent Phi' x passes (compile-time lengths, no grand-potential sums): g.xpers 1 =
// bulk copies two blocks ahead, 2 = per-thread cp.async one block ahead; grid = the row blocks,
// at most the CTAs that fit on the GPU at once.  False if neither applies.
template <typename Real, int N, int NM, typename C>
bool launch_xphi_tma(cudaStream_t st, const GridDesc& g, int LR, const Ctl* ctl, const C* A, const C* B, C* mat,
                     C* phi, float* red_max, int* status, Real kfx, const C* tw) {
    if constexpr (N == 0) {
        return false;
    } else {
        if (!g.xpers || !status) return false;
        const int nsrc = B ? 2 * DFT_NSPEC : DFT_NSPEC;
        const bool cpa = g.xpers == 2;
        const size_t sm = cpa ? dftk::xphi_cpa_smem<Real, N>(NM, LR, nsrc, g.pxh)
                              : dftk::xphi_tma_smem<Real, N>(NM, LR, nsrc, g.pxh);
        static int optin = 0, sms = 0;
        if (optin == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        }
        if (sm > size_t(optin)) return false;
        int occ = 0;
        if (cpa) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_xphi_cpa<Real, N, NM>, dftk::kThreads, sm);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_xphi_tma<Real, N, NM>, dftk::kThreads, sm);
        if (occ < 1) occ = 1;
        const long long nblk = ceil_div((long long)g.ny * g.nz, LR);
        const int grid = (int)(nblk < (long long)sms * occ ? nblk : (long long)sms * occ);
        if (cpa)
            launch_k(dftk::k_xphi_cpa<Real, N, NM>, grid, dftk::kThreads, sm, st, g.pdl, g, LR, ctl, A, B, mat, phi,
                     red_max, status, kfx, tw);
        else
            launch_k(dftk::k_xphi_tma<Real, N, NM>, grid, dftk::kThreads, sm, st, g.pdl, g, LR, ctl, A, B, mat, phi,
                     red_max, status, kfx, tw);
        return true;
    }
}
}  // namespace

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xphi(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl,
                            const C* A, const C* B, C* mat, C* phi, float* red_max, int* status, double* red_phi,
                            Real kfx, const C* tw) {
    if (!red_phi && launch_xphi_tma<Real, N, 1>(st, g, LR, ctl, A, B, mat, phi, red_max, status, kfx, tw))
        return cudaSuccess;
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    launch_k(dftk::k_xphi<Real, N, 1>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, 5 * LR), st, g.pdl, g, px, LR, ctl,
             A, B, mat, phi, red_max, status, red_phi, kfx, tw);
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xphi2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl,
                                    const C* A, const C* B, C* phi, int* status, Real kfx, const C* tw) {
    if (launch_xphi_tma<Real, N, 2>(st, g, LR, ctl, A, B, static_cast<C*>(nullptr), phi, static_cast<float*>(nullptr),
                                    status, kfx, tw))
        return cudaSuccess;
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    launch_k(dftk::k_xphi<Real, N, 2>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, 10 * LR), st, g.pdl,
        g, px, LR, ctl, A, B, nullptr, phi, nullptr, status, nullptr, kfx, tw);
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xupdate(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                               int LR, const Ctl* ctl, const C* cspec, const Real* rho0, const Real* rho1,
                               const Real* V, Real* rho_out, Real* g_out, C* gspec_out, Real* rho_lo,
                               double* red_sum, int* status, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    const int lpr = (sp.S + 1) / 2;
    launch_k(dftk::k_xupdate<Real, N, 1>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, lpr * LR), st, g.pdl,
        g, px, sp, LR, ctl, cspec, nullptr, rho0, rho1, V, rho_out, g_out, gspec_out, rho_lo, red_sum, nullptr,
        status, tw);
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xupdate2(cudaStream_t st, const GridDesc& g, const AxisPlan& px,
                                       const SpeciesDesc<Real>& sp, int LR, const Ctl* ctl, const C* cspec,
                                       const C* cspec2, const Real* rho0, const Real* rho1, const Real* V,
                                       Real* rho_lo, double* red_sum, double* red_sum2, int* status, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    const int lpr = (sp.S + 1) / 2;
    launch_k(dftk::k_xupdate<Real, N, 2>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, 2 * lpr * LR), st, g.pdl,
        g, px, sp, LR, ctl, cspec, cspec2, rho0, rho1, V, nullptr, nullptr, static_cast<C*>(nullptr), rho_lo,
        red_sum, red_sum2, status, tw);
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xinv(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, int ncomp,
                            const C* spec, Real* out, Real* out_last, const Offsets<Real>& off, int cmax,
                            float* red_max, int wd, Real kfx, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    // one component and no outputs: the kernel pairs grid rows in its lines
    const bool rows2 = ncomp == 1 && !wd && !out && !out_last;
    const int lines = rows2 ? (LR + 1) / 2 : (ncomp + 1) / 2 * LR;
    launch_k(dftk::k_xinv<Real, N>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, lines), st, g.pdl,
        g, px, LR, ncomp, spec, out, out_last, off, cmax, red_max, wd, kfx, tw);
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xgrad(cudaStream_t st, const GridDesc& g, const AxisPlan& px,
                                    const SpeciesDesc<Real>& sp, int LR, Real dv, const C* cspec, const Real* rho,
                                    const Real* V, Real* grad_rho, Real* grad_V, double* red, const C* tw) {
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    const int lpr = (sp.S + 1) / 2;
    launch_k(dftk::k_xgrad<Real, N>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, lpr * LR), st, g.pdl,
        g, px, sp, LR, dv, cspec, rho, V, grad_rho, grad_V, red, tw);
    return cudaSuccess;
}

// Lines (species pairs) of the x transform that hold a fixed-number species.
template <typename Real> inline int canon_lines(const SpeciesDesc<Real>& sp, int* lines) {
    int nl = 0;
    for (int l = 0; 2 * l < sp.S; ++l)
        if (sp.canon[2 * l] || (2 * l + 1 < sp.S && sp.canon[2 * l + 1])) lines[nl++] = l;
    return nl;
}

template <typename Real, int N>
cudaError_t LaunchX<Real, N>::xcanon(cudaStream_t st, const GridDesc& g, const AxisPlan& px,
                                     const SpeciesDesc<Real>& sp, int LR, const C* cspec, const Real* V,
                                     double* red, const C* tw) {
    int lines[3] = {0, 0, 0};
    const int nl = canon_lines(sp, lines);
    if (nl == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)ceil_div((long long)g.ny * g.nz, LR);
    launch_k(dftk::k_xcanon<Real, N>, blocks, dftk::kThreads, smem_x_of<C, N>(g.nx, nl * LR), st, g.pdl,
        g, px, sp, LR, nl, lines[0], lines[1], lines[2], cspec, V, red, tw);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------- y
template <typename Real, int N>
cudaError_t LaunchY<Real, N>::init() {
    cudaError_t e = cudaSuccess, r;
    if constexpr (N > 0) {
        constexpr int TY = dft_tile_y<Real>(N);
        if ((r = set_max_smem(dftk::k_yfft_tma<Real, false, N, TY>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_yfft_tma<Real, true, N, TY>)) != cudaSuccess) e = r;
    } else {
        if ((r = set_max_smem(dftk::k_yfft<Real, false, 0, 0>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_yfft<Real, true, 0, 0>)) != cudaSuccess) e = r;
    }
    return e;
}

template <typename Real, int N>
cudaError_t LaunchY<Real, N>::yfft(cudaStream_t st, bool inv, const GridDesc& g, const AxisPlan& py, int T, int ncomp,
                                   C* data, int* status, const C* tw, long long polls) {
    if constexpr (N > 0) {
        // TMA path: persistent CTAs, two TMA-filled stages + one FFT scratch tile + twiddles + 2 mbarriers
        constexpr int TY = dft_tile_y<Real>(N);
        constexpr int E = int(sizeof(C) / 8);
        CUtensorMap map;
        cudaError_t e = tma_encode_3d(&map, data, (unsigned long long)g.nxh * E, (unsigned long long)g.ny,
                                      (unsigned long long)g.nz * ncomp, (unsigned long long)g.pxh * sizeof(C),
                                      (unsigned long long)g.ny * g.pxh * sizeof(C), TY * E, N, 1);
        if (e != cudaSuccess) return e;
        const int ntx = (int)ceil_div(g.nxh, TY);
        const int ntiles = ntx * g.nz * ncomp;
        const size_t sm = dftk::yfft_tma_smem<Real, N, TY>();
        static int per_sm[2] = {0, 0};
        static int sms = 0;
        int& occ = per_sm[inv ? 1 : 0];
        if (occ == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (inv) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_yfft_tma<Real, true, N, TY>, dftk::kThreads, sm);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_yfft_tma<Real, false, N, TY>, dftk::kThreads, sm);
            if (occ < 1) occ = 1;
        }
        const int grid = (int)(ntiles < (long long)sms * occ ? ntiles : sms * occ);
        if (inv) launch_k(dftk::k_yfft_tma<Real, true, N, TY>, grid, dftk::kThreads, sm, st, g.pdl, map, ntx, ntiles, status, tw, polls, 1);
        else launch_k(dftk::k_yfft_tma<Real, false, N, TY>, grid, dftk::kThreads, sm, st, g.pdl, map, ntx, ntiles, status, tw, polls, 1);
        return cudaSuccess;
    } else {
        dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.nz, (unsigned)ncomp);
        const size_t sm = smem_col_of<C>(g.ny, T, 2);
        if (inv) launch_k(dftk::k_yfft<Real, true, 0, 0>, grid, dftk::kThreads, sm, st, g.pdl, g, py, T, data, tw);
        else launch_k(dftk::k_yfft<Real, false, 0, 0>, grid, dftk::kThreads, sm, st, g.pdl, g, py, T, data, tw);
        (void)status;
        (void)polls;
        return cudaSuccess;
    }
}

// ---------------------------------------------------------------------------------- z
// N > 0: grouped kernels (all components of a tile in one transform); N == 0: run-time path.
template <typename Real, int N>
cudaError_t LaunchZ<Real, N>::init() {
    cudaError_t e = cudaSuccess, r;
    if constexpr (N > 0) {
        constexpr int TZ = dft_tile_z<Real>(N);
        if ((r = set_max_smem(dftk::k_zconv_fwd_g<Real, N, TZ, false>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_zconv_fwd_g<Real, N, TZ, true>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_zconv_bwd_g<Real, N, TZ>)) != cudaSuccess) e = r;
        constexpr int TB = dft_tile_zb<Real>(N), TF = dft_tile_zf<Real>(N);
        constexpr int NB = dft_zbwd_threads<Real>(N), MBB = dft_zbwd_minb<Real>(N);
        constexpr int NF = dft_zfwd_threads<Real>(N), MBF = dft_zfwd_minb<Real>(N);
        if constexpr ((TB * sizeof(typename Cplx<Real>::type)) % 16 == 0)
            if ((r = set_max_smem(dftk::k_zconv_bwd_tma<Real, N, TB, NB, MBB>)) != cudaSuccess) e = r;
        if constexpr ((TF * sizeof(typename Cplx<Real>::type)) % 16 == 0) {
            constexpr int MBF3 = dft_zfwd_minb_s3<Real>(N);
            if ((r = set_max_smem(dftk::k_zconv_fwd_tma<Real, N, TF, NF, MBF, DFT_MAXS>)) != cudaSuccess) e = r;
            if ((r = set_max_smem(dftk::k_zconv_fwd_tma<Real, N, TF, NF, MBF3, 3>)) != cudaSuccess) e = r;
        }
        constexpr int TY = dft_tile_y<Real>(N);
        if ((r = set_max_smem(dftk::k_yfft_tma<Real, false, N, TY, true>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_yfft_tma<Real, true, N, TY, true>)) != cudaSuccess) e = r;
    } else {
        if ((r = set_max_smem(dftk::k_zconv_fwd<Real, 0, 0, false>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_zconv_fwd<Real, 0, 0, true>)) != cudaSuccess) e = r;
        if ((r = set_max_smem(dftk::k_zconv_bwd<Real, 0, 0>)) != cudaSuccess) e = r;
    }
    return e;
}

template <typename Real, int N>
cudaError_t LaunchZ<Real, N>::zfft(cudaStream_t st, bool inv, const GridDesc& g, int ncomp, C* data, int* status,
                                   const C* tw, long long polls) {
    if constexpr (N > 0) {
        // the y pass's persistent TMA kernel along z: tiles of TY kx columns x nz at one ky
        constexpr int TY = dft_tile_y<Real>(N);
        constexpr int E = int(sizeof(C) / 8);
        CUtensorMap map;
        cudaError_t e = tma_encode_3d(&map, data, (unsigned long long)g.nxh * E, (unsigned long long)g.ny,
                                      (unsigned long long)g.nz * ncomp, (unsigned long long)g.pxh * sizeof(C),
                                      (unsigned long long)g.ny * g.pxh * sizeof(C), TY * E, 1, N);
        if (e != cudaSuccess) return e;
        const int ntx = (int)ceil_div(g.nxh, TY);
        const int ntiles = ntx * g.ny * ncomp;
        const size_t sm = dftk::yfft_tma_smem<Real, N, TY>();
        static int per_sm[2] = {0, 0};
        static int sms = 0;
        int& occ = per_sm[inv ? 1 : 0];
        if (occ == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (inv) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_yfft_tma<Real, true, N, TY, true>, dftk::kThreads, sm);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_yfft_tma<Real, false, N, TY, true>, dftk::kThreads, sm);
            if (occ < 1) occ = 1;
        }
        const int grid = (int)(ntiles < (long long)sms * occ ? ntiles : sms * occ);
        if (inv)
            return launch_k(dftk::k_yfft_tma<Real, true, N, TY, true>, grid, dftk::kThreads, sm, st, g.pdl, map, ntx,
                            ntiles, status, tw, polls, g.ny);
        return launch_k(dftk::k_yfft_tma<Real, false, N, TY, true>, grid, dftk::kThreads, sm, st, g.pdl, map, ntx,
                        ntiles, status, tw, polls, g.ny);
    } else {
        (void)st; (void)inv; (void)g; (void)ncomp; (void)data; (void)status; (void)tw; (void)polls;
        return cudaErrorNotSupported;
    }
}

template <typename Real, int N>
cudaError_t LaunchZ<Real, N>::zconv_fwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                                 int T, Real kfx, Real kfy, Real kfz, int want_psi, const C* in, C* slot_n,
                                 C* slot_es, double* red_energy, const C* tw, int* status) {
    constexpr int TZ = N > 0 ? dft_tile_z<Real>(N) : 1;
    constexpr int TB = N > 0 ? dft_tile_zf<Real>(N) : 1;
    constexpr bool kTma = N > 0 && (TB * sizeof(C)) % 16 == 0;
    if constexpr (kTma) {
        static int optin = 0, sms = 0;
        if (optin == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        }
        const size_t sm = dftk::zfwd_tma_smem<Real, N, TB>(sp.S);
        if (!red_energy && status && !g.zgrp && sm <= size_t(optin)) {
            // TMA path (the grand-potential sums keep the one-tile-per-CTA kernel below)
            constexpr int NT = dft_zfwd_threads<Real>(N), MB = dft_zfwd_minb<Real>(N);
            constexpr int E = int(sizeof(C) / 8);
            CUtensorMap map_in, map_n;
            auto encode = [&](CUtensorMap* m, const C* data, int ncomp) {
                return tma_encode_3d(m, const_cast<C*>(data), (unsigned long long)g.nxh * E, (unsigned long long)g.ny,
                                     (unsigned long long)g.nz * ncomp, (unsigned long long)g.pxh * sizeof(C),
                                     (unsigned long long)g.ny * g.pxh * sizeof(C), TB * E, 1, N);
            };
            cudaError_t e = encode(&map_in, in, sp.S);
            if (e == cudaSuccess) e = encode(&map_n, slot_n, DFT_NSPEC);
            if (e != cudaSuccess) return e;
            const int ntx = (int)ceil_div(g.nxh, TB);
            const int ntiles = ntx * g.ny;
            // at most three species: the instance whose records and species loops are sized for three
            constexpr int MB3 = dft_zfwd_minb_s3<Real>(N);
            auto kern = sp.S <= 3 ? dftk::k_zconv_fwd_tma<Real, N, TB, NT, MB3, 3>
                                  : dftk::k_zconv_fwd_tma<Real, N, TB, NT, MB, DFT_MAXS>;
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, sm);
            if (occ < 1) occ = 1;
            const int grid = (int)(ntiles < (long long)sms * occ ? ntiles : sms * occ);
            launch_k(kern, grid, NT, sm, st, g.pdl, map_in, map_n, g, sp, kfx, kfy, kfz, want_psi, slot_es, ntx, ntiles,
                     status, tw);
            return cudaSuccess;
        }
    }
    if constexpr (N > 0) {
        const size_t sm = dftk::zg_smem_bytes<TZ, N>(sizeof(C));
        dim3 grid((unsigned)ceil_div(g.nxh, TZ), (unsigned)g.ny);
        if (red_energy)
            launch_k(dftk::k_zconv_fwd_g<Real, N, TZ, true>, grid, dftk::kThreads, sm, st, g.pdl,
                g, sp, kfx, kfy, kfz, want_psi, in, slot_n, slot_es, red_energy, tw);
        else
            launch_k(dftk::k_zconv_fwd_g<Real, N, TZ, false>, grid, dftk::kThreads, sm, st, g.pdl,
                g, sp, kfx, kfy, kfz, want_psi, in, slot_n, slot_es, nullptr, tw);
    } else {
        dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.ny);
        const size_t sm = smem_col_of<C>(g.nz, T, 7);
        if (red_energy)
            launch_k(dftk::k_zconv_fwd<Real, 0, 0, true>, grid, dftk::kThreads, sm, st, g.pdl,
                g, pz, sp, T, kfx, kfy, kfz, want_psi, in, slot_n, slot_es, red_energy, tw);
        else
            launch_k(dftk::k_zconv_fwd<Real, 0, 0, false>, grid, dftk::kThreads, sm, st, g.pdl,
                g, pz, sp, T, kfx, kfy, kfz, want_psi, in, slot_n, slot_es, nullptr, tw);
    }
    return cudaSuccess;
}

namespace {
// The persistent TMA second-half z pass: single (pair = 0: nine Phi' spectra at phi, results over
// its first ncomp_out) or the two line-search samples (pair = 1: eighteen at phi, weights in
// ctl[0], ctl[1], results at phi components 0 .. 2 ncomp_out - 1).  False if it does not apply
// (no compile-time length, the grouped variant chosen, or too little shared memory).
template <typename Real, int N, typename C>
bool launch_zbwd_tma(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx, Real kfy, Real kfz,
                     int flags, int ncomp_out, int pair, const Ctl* ctl, C* phi, const C* esA, const C* esB, C* es_mat,
                     const C* tw) {
    constexpr int TB = N > 0 ? dft_tile_zb<Real>(N) : 1;
    constexpr bool kTma = N > 0 && (TB * sizeof(C)) % 16 == 0;
    if constexpr (!kTma) {
        return false;
    } else {
        const bool es_on = (flags & 2) != 0;
        const int nes = es_on ? ncomp_out * (esB ? 2 : 1) : 0;
        static int optin = 0, sms = 0;
        if (optin == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        }
        const size_t sm = dftk::zbwd_tma_smem<Real, N, TB>(nes);
        if (g.zgrp || sm > size_t(optin)) return false;
        // persistent CTAs, two TMA-filled stages of nine Phi' tiles, one area of ES tiles
        constexpr int NT = dft_zbwd_threads<Real>(N), MB = dft_zbwd_minb<Real>(N);
        constexpr int E = int(sizeof(C) / 8);
        CUtensorMap map_phi, map_esA, map_esB, map_out;
        auto encode = [&](CUtensorMap* m, const C* data, int ncomp) {
            return tma_encode_3d(m, const_cast<C*>(data), (unsigned long long)g.nxh * E, (unsigned long long)g.ny,
                                 (unsigned long long)g.nz * ncomp, (unsigned long long)g.pxh * sizeof(C),
                                 (unsigned long long)g.ny * g.pxh * sizeof(C), TB * E, 1, N);
        };
        const int nphi = (pair ? 2 : 1) * DFT_NSPEC;
        cudaError_t e = encode(&map_phi, phi, nphi);
        if (e == cudaSuccess) e = encode(&map_esA, es_on ? esA : phi, es_on ? ncomp_out : DFT_NSPEC);
        if (e == cudaSuccess) e = encode(&map_esB, (es_on && esB) ? esB : phi, (es_on && esB) ? ncomp_out : DFT_NSPEC);
        if (e == cudaSuccess) e = encode(&map_out, phi, nphi);
        if (e != cudaSuccess) return false;
        const int ntx = (int)ceil_div(g.nxh, TB);
        const int ntiles = ntx * g.ny;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dftk::k_zconv_bwd_tma<Real, N, TB, NT, MB>, NT, sm);
        if (occ < 1) occ = 1;
        const int grid = (int)(ntiles < (long long)sms * occ ? ntiles : sms * occ);
        // the status word of the device control block records a TMA wait that ran out
        int* status = const_cast<int*>(&ctl->status);
        launch_k(dftk::k_zconv_bwd_tma<Real, N, TB, NT, MB>, grid, NT, sm, st, g.pdl, map_phi, map_esA, map_esB,
                 map_out, g, sp, kfx, kfy, kfz, flags, ncomp_out, esB ? 1 : 0, pair, ctl, es_mat, ntx, ntiles, status,
                 tw);
        return true;
    }
}
}  // namespace

template <typename Real, int N>
cudaError_t LaunchZ<Real, N>::zconv_bwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                                 int T, Real kfx, Real kfy, Real kfz, int flags, int ncomp_out, const Ctl* ctl, C* phi,
                                 const C* esA, const C* esB, C* es_mat, const C* tw) {
    constexpr int TZ = N > 0 ? dft_tile_z<Real>(N) : 1;
    if (launch_zbwd_tma<Real, N>(st, g, sp, kfx, kfy, kfz, flags, ncomp_out, 0, ctl, phi, esA, esB, es_mat, tw))
        return cudaSuccess;
    if constexpr (N > 0) {
        const size_t sm = dftk::zg_smem_bytes<TZ, N>(sizeof(C));
        dim3 grid((unsigned)ceil_div(g.nxh, TZ), (unsigned)g.ny);
        launch_k(dftk::k_zconv_bwd_g<Real, N, TZ>, grid, dftk::kThreads, sm, st, g.pdl,
            g, sp, kfx, kfy, kfz, flags, ncomp_out, ctl, phi, esA, esB, es_mat, tw);
    } else {
        dim3 grid((unsigned)ceil_div(g.nxh, T), (unsigned)g.ny);
        launch_k(dftk::k_zconv_bwd<Real, 0, 0>, grid, dftk::kThreads, smem_col_of<C>(g.nz, T, 7), st, g.pdl,
            g, pz, sp, T, kfx, kfy, kfz, flags, ncomp_out, ctl, phi, esA, esB, es_mat, tw);
    }
    return cudaSuccess;
}

template <typename Real, int N>
cudaError_t LaunchZ<Real, N>::zconv_bwd_pair(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx,
                                             Real kfy, Real kfz, int ncomp_out, const Ctl* ctl, C* phi, const C* esA,
                                             const C* esB, const C* tw) {
    if (launch_zbwd_tma<Real, N>(st, g, sp, kfx, kfy, kfz, 3, ncomp_out, 1, ctl, phi, esA, esB,
                                 static_cast<C*>(nullptr), tw))
        return cudaSuccess;
    return cudaErrorNotSupported;
}

template <typename Real, int N>
bool LaunchZ<Real, N>::has_zbwd_pair(const GridDesc& g, int ncomp_out) {
    constexpr int TB = N > 0 ? dft_tile_zb<Real>(N) : 1;
    if constexpr (N > 0 && (TB * sizeof(C)) % 16 == 0) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return !g.zgrp && dftk::zbwd_tma_smem<Real, N, TB>(2 * ncomp_out) <= size_t(optin);
    } else {
        return false;
    }
}
