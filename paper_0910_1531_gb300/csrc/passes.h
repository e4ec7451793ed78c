// Host-side launchers of the pass kernels.
//
// Passes<Real> is the interface the plan code calls; it dispatches on the axis length to
// LaunchX / LaunchY / LaunchZ<Real, N>, whose kernels have the transform length N (and the
// column tile width) fixed at compile time.  N = 0 is the run-time path for any length.
// Each (Real, N) pair is compiled in its own translation unit (kinst.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

// Axis lengths with compile-time kernels.
#define DFT_CT_SIZES(X) X(32) X(48) X(64) X(96) X(128) X(256)

__host__ __device__ constexpr bool dft_is_ct_size(int n) {
    return n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 256;
}

// Column-tile widths of the compile-time y and z passes (kx columns per tile).
#ifndef DFT_TILE_Y_SHIFT
#define DFT_TILE_Y_SHIFT 0
#endif
template <typename Real> __host__ __device__ constexpr int dft_tile_y(int n) {
    return (sizeof(Real) == 4 ? 16 : 8) >> DFT_TILE_Y_SHIFT;
}
// The compile-time z passes transform all components of a tile together (two pools of ten
// tiles in shared memory): the width keeps a CTA near 86 KB (FP32) so that two fit on an SM.
// DFT_TILE_ZG_SHIFT (build flag, default 0) narrows the tiles by that power of two.
#ifndef DFT_TILE_ZG_SHIFT
#define DFT_TILE_ZG_SHIFT 0
#endif
template <typename Real> __host__ __device__ constexpr int dft_tile_z(int n) {
    const int t = (n <= 32 ? 16 : (n <= 64 ? 8 : (n <= 128 ? 4 : 2))) / (sizeof(Real) == 4 ? 1 : 2);
    return (t >> DFT_TILE_ZG_SHIFT) > 0 ? (t >> DFT_TILE_ZG_SHIFT) : 1;
}

// Persistent TMA z passes: half the grouped width (at least 16 bytes of a row, the TMA
// minimum).
template <typename Real> __host__ __device__ constexpr int dft_tile_zb(int n) {
    const int t = dft_tile_z<Real>(n) / 2, tmin = sizeof(Real) == 4 ? 2 : 1;
    return t > tmin ? t : tmin;
}
// Tile width of the persistent TMA first-half z pass: the second half's (DFT_ZFWD_WIDE: the
// grouped width).
template <typename Real> __host__ __device__ constexpr int dft_tile_zf(int n) {
#ifdef DFT_ZFWD_WIDE
    return dft_tile_z<Real>(n);
#else
    return dft_tile_zb<Real>(n);
#endif
}

// Threads of the persistent TMA z passes and the resident CTAs per SM their register budget
// is sized for.  First half: 256 threads, two CTAs per SM, up to length 128; 512 threads, one
// CTA, at 256.  Second half: 256 threads, three CTAs per SM (FP32; two in FP64, whose
// butterflies need twice the registers), up to 128; 288 threads (nine warps: one pass of the
// threads covers the radix-16 butterflies of the nine Phi' groups of a two-column tile), two
// CTAs per SM, at 256 (its shared memory allows no more).  DFT_ZFWD_THREADS / DFT_ZFWD_MINB / DFT_ZBWD_THREADS / DFT_ZBWD_MINB (build
// flags) override.
template <typename Real> __host__ __device__ constexpr int dft_zfwd_threads(int n) {
#ifdef DFT_ZFWD_THREADS
    return DFT_ZFWD_THREADS;
#else
    return n >= 256 ? 512 : 256;
#endif
}
template <typename Real> __host__ __device__ constexpr int dft_zfwd_minb(int n) {
#ifdef DFT_ZFWD_MINB
    return DFT_ZFWD_MINB;
#else
    return dft_zfwd_threads<Real>(n) <= 256 ? 2 : 1;
#endif
}
// The first-half pass for at most three species (its table records and species loops sized for
// three): resident CTAs per SM its register budget is sized for (DFT_ZFWD_MINB_S3 overrides).
template <typename Real> __host__ __device__ constexpr int dft_zfwd_minb_s3(int n) {
#ifdef DFT_ZFWD_MINB_S3
    return DFT_ZFWD_MINB_S3;
#else
    return dft_zfwd_minb<Real>(n);
#endif
}
template <typename Real> __host__ __device__ constexpr int dft_zbwd_threads(int n) {
#ifdef DFT_ZBWD_THREADS
    return DFT_ZBWD_THREADS;
#else
    return n >= 256 ? 288 : 256;
#endif
}
template <typename Real> __host__ __device__ constexpr int dft_zbwd_minb(int n) {
#ifdef DFT_ZBWD_MINB
    return DFT_ZBWD_MINB;
#else
    return (n < 256 && sizeof(Real) == 4) ? 3 : 2;
#endif
}

template <typename Real, int N>
struct LaunchX {
    using C = typename Cplx<Real>::type;
    static cudaError_t init();
    static cudaError_t xfwd(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int ncomp, int lx, const Real* in,
                     C* out, const C* tw);
    static cudaError_t xphi(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl, const C* A,
                     const C* B, C* mat, C* phi, float* red_max, int* status, double* red_phi, Real kfx,
                     const C* tw);
    static cudaError_t xupdate(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp, int LR,
                        const Ctl* ctl, const C* cspec, const Real* rho0, const Real* rho1, const Real* V,
                        Real* rho_out, Real* g_out, C* gspec_out, Real* rho_lo, double* red_sum, int* status,
                        const C* tw);
    // the two line-search samples in one pass each (weights from ctl[1] and ctl[2]): Phi' of
    // both mixtures of the slots (sample m's nine spectra at phi + m DFT_NSPEC nc), and the
    // update pass's residual sums of both (c spectra at cspec / cspec2, sums into red_sum /
    // red_sum2; nothing written to rho or G)
    static cudaError_t xphi2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl,
                             const C* A, const C* B, C* phi, int* status, Real kfx, const C* tw);
    static cudaError_t xupdate2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                                int LR, const Ctl* ctl, const C* cspec, const C* cspec2, const Real* rho0,
                                const Real* rho1, const Real* V, Real* rho_lo, double* red_sum, double* red_sum2,
                                int* status, const C* tw);
    static cudaError_t xinv(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, int ncomp, const C* spec,
                     Real* out, Real* out_last, const Offsets<Real>& off, int cmax, float* red_max, int wd,
                     Real kfx, const C* tw);
    static cudaError_t xgrad(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                             int LR, Real dv, const C* cspec, const Real* rho, const Real* V, Real* grad_rho,
                             Real* grad_V, double* red, const C* tw);
    static cudaError_t xcanon(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                              int LR, const C* cspec, const Real* V, double* red, const C* tw);
};

template <typename Real, int N>
struct LaunchY {
    using C = typename Cplx<Real>::type;
    static cudaError_t init();
    static cudaError_t yfft(cudaStream_t st, bool inv, const GridDesc& g, const AxisPlan& py, int T, int ncomp, C* data,
                     int* status, const C* tw, long long polls);
};

template <typename Real, int N>
struct LaunchZ {
    using C = typename Cplx<Real>::type;
    static cudaError_t init();
    static cudaError_t zconv_fwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp, int T,
                          Real kfx, Real kfy, Real kfz, int want_psi, const C* in, C* slot_n, C* slot_es,
                          double* red_energy, const C* tw, int* status);
    static cudaError_t zconv_bwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp, int T,
                          Real kfx, Real kfy, Real kfz, int flags, int ncomp_out, const Ctl* ctl, C* phi,
                          const C* esA, const C* esB, C* es_mat, const C* tw);
    static cudaError_t zconv_bwd_pair(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx,
                                      Real kfy, Real kfz, int ncomp_out, const Ctl* ctl, C* phi, const C* esA,
                                      const C* esB, const C* tw);
    static bool has_zbwd_pair(const GridDesc& g, int ncomp_out);
    static cudaError_t zfft(cudaStream_t st, bool inv, const GridDesc& g, int ncomp, C* data, int* status,
                            const C* tw, long long polls);
};

template <typename Real>
struct Passes {
    using C = typename Cplx<Real>::type;
    static cudaError_t init_attributes();
    // dynamic shared memory of an x pass with `lines` lines and of a column pass with nbuf tiles
    static size_t smem_x(int nx, int lines) { return (size_t(nx) + 2 * size_t(lines) * (nx + 1)) * sizeof(C) + 16; }
    static size_t smem_col(int n, int T, int nbuf) { return (size_t(n) + size_t(nbuf) * T * n) * sizeof(C) + 16; }
    // tile widths: the compile-time value for specialised lengths, else the largest that fits `budget`
    static int tile_y(int n, size_t budget);
    static int tile_z(int n, size_t budget);

    static cudaError_t xfwd(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int ncomp, int lx, const Real* in,
                     C* out, const C* tw);
    // polls: bound of each TMA tile wait (DFT_WAIT_POLLS; the drains after a give-up keep it)
    static cudaError_t yfft(cudaStream_t st, bool inv, const GridDesc& g, const AxisPlan& py, int T, int ncomp, C* data,
                     int* status, const C* tw, long long polls = DFT_WAIT_POLLS);
    static cudaError_t zconv_fwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp, int T,
                          Real kfx, Real kfy, Real kfz, int want_psi, const C* in, C* slot_n, C* slot_es,
                          double* red_energy, const C* tw, int* status);
    static cudaError_t xphi(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl, const C* A,
                     const C* B, C* mat, C* phi, float* red_max, int* status, double* red_phi, Real kfx,
                     const C* tw);
    static cudaError_t zconv_bwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp, int T,
                          Real kfx, Real kfy, Real kfz, int flags, int ncomp_out, const Ctl* ctl, C* phi,
                          const C* esA, const C* esB, C* es_mat, const C* tw);
    // The two line-search samples' second-half z passes in one launch (both hard-sphere and ES
    // parts): phi holds sample 1's nine Phi' spectra then sample 2's, ctl[0] / ctl[1] their
    // weights; sample m's ncomp_out results go to phi components m ncomp_out ...  Only where
    // has_zbwd_pair (the persistent TMA pass); cudaErrorNotSupported otherwise.
    static cudaError_t zconv_bwd_pair(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx,
                                      Real kfy, Real kfz, int ncomp_out, const Ctl* ctl, C* phi, const C* esA,
                                      const C* esB, const C* tw);
    static bool has_zbwd_pair(const GridDesc& g, int ncomp_out);
    // The split first-half z stage (compile-time lengths): zfft = the persistent TMA z transform
    // of ncomp components in place (tiles of the y pass's width; cudaErrorNotSupported for other
    // lengths), zmul = the k-space products from the S species spectra into the nine
    // weighted-density spectra (slot_n, 1/N applied) and the S ES spectra (slot_es).
    static cudaError_t zfft(cudaStream_t st, bool inv, const GridDesc& g, int ncomp, C* data, int* status,
                            const C* tw, long long polls);
    static cudaError_t zmul(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx, Real kfy,
                            Real kfz, const C* in, C* slot_n, C* slot_es);
    // rho_lo (or nullptr): low part of an extended iterate rho0 + rho_lo, read
    // with rho0 and, when rho_out is written, replaced by the low part of the new iterate;
    // gspec_out (or nullptr): also the x half spectra of G (S components, the layout of xfwd's
    // output), the next first half's input
    static cudaError_t xupdate(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp, int LR,
                        const Ctl* ctl, const C* cspec, const Real* rho0, const Real* rho1, const Real* V,
                        Real* rho_out, Real* g_out, C* gspec_out, Real* rho_lo, double* red_sum, int* status,
                        const C* tw);
    // the two line-search samples in one pass each (weights from ctl[1] and ctl[2]): Phi' of
    // both mixtures of the slots (sample m's nine spectra at phi + m DFT_NSPEC nc), and the
    // update pass's residual sums of both (c spectra at cspec / cspec2, sums into red_sum /
    // red_sum2; nothing written to rho or G)
    static cudaError_t xphi2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl,
                             const C* A, const C* B, C* phi, int* status, Real kfx, const C* tw);
    static cudaError_t xupdate2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                                int LR, const Ctl* ctl, const C* cspec, const C* cspec2, const Real* rho0,
                                const Real* rho1, const Real* V, Real* rho_lo, double* red_sum, double* red_sum2,
                                int* status, const C* tw);
    static cudaError_t xinv(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, int ncomp, const C* spec,
                     Real* out, Real* out_last, const Offsets<Real>& off, int cmax, float* red_max, int wd,
                     Real kfx, const C* tw);
    static cudaError_t xgrad(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                             int LR, Real dv, const C* cspec, const Real* rho, const Real* V, Real* grad_rho,
                             Real* grad_V, double* red, const C* tw);
    // sums for the normalisation of fixed-number species (red: [blocks][DFT_MAXS]) and the
    // scale factors they give (into ctl->canon_scale)
    static cudaError_t xcanon(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                              int LR, const C* cspec, const Real* V, double* red, const C* tw);
    static cudaError_t canon_scale(cudaStream_t st, Ctl* ctl, const SpeciesDesc<Real>& sp, const double* red,
                                   int nblocks, int pdl);
    // fill the |k| tables of sp (tab_w, tab_k, tab_dk, tab_m2max set by the caller) for wave
    // number kf of a cubic box
    static cudaError_t build_ktab(cudaStream_t st, const SpeciesDesc<Real>& sp, double kf);
    // fill out[nx + ny + nz] with the per-axis Laplacian terms of grid g (SpeciesDesc::lap1d)
    static cudaError_t build_laptab(cudaStream_t st, const GridDesc& g, Real kfx, Real kfy, Real kfz, Real* out);
};

// ctl: the plan's three control blocks (iteration, sample 1 weights, sample 2 weights);
// red_sum2 (or nullptr): the second sample's partial sums for FIN_F12_CHOOSE; pdl: launch with
// programmatic dependent launch (GridDesc::pdl)
cudaError_t launch_finalize(cudaStream_t st, Ctl* ctl, const double* red_sum, const double* red_sum2, int nsum,
                            const float* red_max, int nmax, int op, double inv_count, double alpha_fixed,
                            double n3_bound, double alpha_floor, int pdl);

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
