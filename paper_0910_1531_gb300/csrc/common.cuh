// Shared definitions of the GB300 classical-DFT kernels: complex arithmetic,
// per-axis FFT plans, grid / species descriptors and the device control block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "gb300dft.h"

#define DFT_MAXS 5          // species (the back-convolution keeps 5 k-space accumulators)
#define DFT_MAXSTAGES 8     // radix stages per axis
#define DFT_NCOMP 10        // n0 n1 n2 n3 nV1(xyz) nV2(xyz)
// Weighted-density spectra kept between the passes: n0 n1 n2 n3, m (n_V1 = grad m), then
// i k_y m, i k_z m, i k_y n3, i k_z n3.  The x components i k_x m and i k_x n3 are formed in
// the x pass that takes the spectra to real space (and the divergence terms of the back
// convolution in the x pass that leaves it), so the y and z passes carry nine components.
#define DFT_NSPEC 9
// Polls of a TMA tile wait before it gives up (the plans' default; dft_set_wait_polls)
#define DFT_WAIT_POLLS (1LL << 24)

template <typename Real> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C().x) re, decltype(C().x) im) {
    C c; c.x = re; c.y = im; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C().x) s) { return cmake<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
// multiply by +i or -i
template <typename C> __device__ __forceinline__ C cmul_i(C a) { return cmake<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }

// Radix decomposition of one axis length: n = prod radix[s]; radices 2, 3, 4, 8, 16 and the
// odd primes 5..DFT_MAX_PRIME (run-time transforms only; see dft_radix_plan).
struct AxisPlan {
    int n;
    int nstages;
    int radix[DFT_MAXSTAGES];
};

// Largest prime factor an axis length may have.  Factors 5..31 take a direct odd-radix stage
// (the R-point DFT by its definition) in the run-time transforms.
#define DFT_MAX_PRIME 31

// Radix plan of an axis length: the 3s, then the other odd primes up to DFT_MAX_PRIME, then
// 16s and one of 2 / 4 / 8.  False if n has a larger prime factor or needs more than
// DFT_MAXSTAGES stages.
inline bool dft_radix_plan(int n, AxisPlan* out) {
    out->n = n;
    out->nstages = 0;
    int m = n;
    auto push = [&](int r) {
        if (out->nstages >= DFT_MAXSTAGES) return false;
        out->radix[out->nstages++] = r;
        return true;
    };
    while (m % 3 == 0) { if (!push(3)) return false; m /= 3; }
    for (int p = 5; p <= DFT_MAX_PRIME; p += 2)
        while (m % p == 0) { if (!push(p)) return false; m /= p; }
    while (m >= 16 && m % 16 == 0) { if (!push(16)) return false; m /= 16; }
    if (m == 2 || m == 4 || m == 8) { if (!push(m)) return false; m = 1; }
    return m == 1 && out->nstages > 0;
}

// Axis lengths a plan accepts: 4 <= n <= 512 with a radix plan.
inline bool dft_valid_length(int n) {
    AxisPlan p;
    return n >= 4 && n <= 512 && dft_radix_plan(n, &p);
}

// Grid of one state point.  Real fields: [c][nz][ny][nx]; half spectra after the
// x transform: [c][nz][ny][pxh], of which kx < nxh = nx/2 + 1 are used; the row pitch
// pxh is nxh rounded up to even so that every row starts on a 16-byte boundary (a TMA
// requirement).
struct GridDesc {
    int nx, ny, nz, nxh, pxh;
    long long n;     // nx * ny * nz
    long long nc;    // nz * ny * pxh (elements per half-spectrum component)
    double hx, hy, hz;
    int phi;         // hard-sphere free-energy density of the state point (DFT_PHI_*; 0 = eq. Phi)
    // transform variants chosen by the autotuner (0 for all: the compile-time passes where a
    // length has them): x passes by the run-time kernels with the plan's AxisPlan; y passes by
    // the run-time column kernel; z passes by the one-tile-per-CTA grouped kernels instead of
    // the persistent TMA ones
    int xrt, yrt, zgrp;
    int xpers;       // the Phi' x passes as a persistent kernel: 1 bulk-copy prefetch, 2 cp.async prefetch
    int zsplit;      // the first-half z stage as three passes: z transform, k-space products, z transform
    int pdl;         // launch the passes with programmatic dependent launch (launch_k)
};

// Programmatic dependent launch.  With GridDesc::pdl set the passes are launched with the
// programmatic-stream-serialization attribute, so that the launch of one pass overlaps the
// completion of the previous one.  dep_wait() (griddepcontrol.wait) returns once every grid
// the kernel depends on has completed and its memory writes are visible; each pass calls it
// before its first access to memory an earlier kernel may write (for a kernel launched without
// the attribute it returns at once).  dep_launch() (griddepcontrol.launch_dependents) lets the
// next kernel be scheduled once every CTA of this one has issued it or exited.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Where a pass lets the next one be scheduled (build flag): 0 (default) = never, the next pass
// is scheduled as this one's CTAs exit (its launch still overlaps this one's completion); 1 = at
// its start.  Measured on the 128^3 iteration: 0 runs 0.5 % faster than plain stream order, 1
// 13 % slower (the next pass's waiting CTAs become resident beside the persistent passes).
#ifndef DFT_DEP_TRIGGER
#define DFT_DEP_TRIGGER 0
#endif
__device__ __forceinline__ void dep_launch() {
#if DFT_DEP_TRIGGER
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Launch `kernel` on `st`, with the programmatic-serialization attribute when pdl != 0.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int pdl,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Species constants in the kernels' precision (host fills them in double, then converts).
template <typename Real>
struct SpeciesDesc {
    int S;
    Real R[DFT_MAXS];
    Real z[DFT_MAXS];
    Real rho_b[DFT_MAXS];
    Real inv_rho_b[DFT_MAXS];   // residual weights 1 / rho_bath
    Real mu_hs_b[DFT_MAXS];     // beta mu^{HS,bath}
    Real mu_ex_b[DFT_MAXS];     // beta mu^{ex,bath} = beta (mu^{HS,bath} + mu^{ES,bath})
    Real n_rho_b[DFT_MAXS];     // N * rho_bath: DFT of the bath density at k = 0
    // bulk-fluid kernel per pair (i, j), in kT units
    Real es_pref[DFT_MAXS][DFT_MAXS];   // lambda_B z_i z_j / 2
    Real es_a[DFT_MAXS][DFT_MAXS];      // 1 / (2 l_i l_j)
    Real es_b[DFT_MAXS][DFT_MAXS];      // (l_i + l_j) / (l_i l_j)
    Real es_c[DFT_MAXS][DFT_MAXS];      // (l_i - l_j)^2 / (2 l_i l_j) + 2
    Real es_R[DFT_MAXS][DFT_MAXS];      // R_ij = R_i + R_j
    Real pois[DFT_MAXS][DFT_MAXS];      // 4 pi lambda_B z_i z_j
    Real es_da[DFT_MAXS][DFT_MAXS];     // d es_a / d Gamma  (gradient with respect to the bath)
    Real es_db[DFT_MAXS][DFT_MAXS];     // d es_b / d Gamma
    Real es_dc[DFT_MAXS][DFT_MAXS];     // d es_c / d Gamma
    Real inv_n;                         // 1 / N
    int coulomb_limit;                  // Gamma == 0: kernel is lambda_B z_i z_j / r inside R_ij
    // Optional tables of the |k|-only factors on a cubic box, indexed by the integer
    // m2 = mx^2 + my^2 + mz^2 (|k| = kf sqrt(m2)); null: the kernels evaluate them per point.
    const Real* tab_w;                  // [m2][tab_ws]: w0_s at 2 s, j3_s at 2 s + 1
    const Real* tab_k;                  // [m2][tab_ks]: DC_ij_hat at j (j + 1) / 2 + i, i <= j
    const Real* tab_dk;                 // [m2][tab_ks]: d DC_ij_hat / d Gamma, same order
    int tab_m2max;
    int tab_ws, tab_ks;                 // record lengths: 2 S and S (S + 1) / 2 rounded up to 16 bytes
    // Optional per-axis terms of the discrete Laplacian, sin^2(k_d h_d / 2) / h_d^2 by FFT index:
    // x indices at 0, y at nx, z at nx + ny (k_laptab); null: the kernels evaluate them per point.
    const Real* lap1d;
    // fixed-number species (canonical form of eq. rhoEquation): canon[i] != 0, target sum of G_i
    // over the grid N_i / h^3; ncanon of them
    int canon[DFT_MAXS];
    double nfix_dv[DFT_MAXS];
    int ncanon;
};

// Index of the pair (i, j), i <= j, in a table record (independent of S).
__host__ __device__ constexpr int dft_pair(int i, int j) { return j * (j + 1) / 2 + i; }

// Register capacity of a table record (a multiple of 16 bytes of either precision).
#define DFT_TAB_W 12        // >= 2 DFT_MAXS
#define DFT_TAB_K 16        // >= DFT_MAXS (DFT_MAXS + 1) / 2

// Per-component additive constants of the plain x inverse.
template <typename Real> struct Offsets { Real v[DFT_NCOMP + 2]; };

// Device-resident control block of the Picard iteration.  Kernels read the mixing
// weights from here, so a whole iteration can be queued (or captured) without a
// host round trip.
struct Ctl {
    double wA, wB;          // weights of slot A / slot B weighted densities (XPHI, ZK2)
    double w0, w1;          // weights of rho^(0) / rho^(1) (XU)
    double f[4];            // squared residuals: f0 = r^2(rho0), f1, f2 samples, f3 = accepted point
    double alpha_max;       // n3 bound of the step
    double alpha_s;         // sampled interval min(alpha_max, 2 alpha_prev)
    double alpha;           // accepted alpha of the last step (alpha_prev of the next)
    double alpha_fixed;     // < 0: line search
    double n3max_cur;       // max n3 of the current iterate
    double n3max_next;      // max n3 of G(current)
    double resid;           // sqrt(f0)
    double resid_prev;      // r of the iterate a step started from
    double sample_alpha[2];
    int status;             // dft_status bits raised on the device (see DEV_* below)
    int iter;
    int loop_left;          // iterations left in an on-device loop of dft_iter_run / dft_batch_iterate
    // fixed-number species: G_i = canon_scale[i] exp(-V_i + c_i), canon_scale = N_i / (h^3 sum e)
    double canon_scale[DFT_MAXS];
    // the four weights rounded to float when they are set: the FP32 passes read these, since a
    // double-to-float conversion in every thread queues on the narrow FP64 pipe
    float wAf, wBf, w0f, w1f;
};

// The weights of a control block in the working precision.
template <typename Real> struct CtlW;
template <> struct CtlW<float> {
    static __device__ __forceinline__ float wA(const Ctl* c) { return c->wAf; }
    static __device__ __forceinline__ float wB(const Ctl* c) { return c->wBf; }
    static __device__ __forceinline__ float w0(const Ctl* c) { return c->w0f; }
    static __device__ __forceinline__ float w1(const Ctl* c) { return c->w1f; }
};
template <> struct CtlW<double> {
    static __device__ __forceinline__ double wA(const Ctl* c) { return c->wA; }
    static __device__ __forceinline__ double wB(const Ctl* c) { return c->wB; }
    static __device__ __forceinline__ double w0(const Ctl* c) { return c->w0; }
    static __device__ __forceinline__ double w1(const Ctl* c) { return c->w1; }
};

enum {
    DEV_N3BOUND = 1,        // n3 >= 1 met
    DEV_NONFINITE = 2,      // non-finite density or residual met
    DEV_TIMEOUT = 4         // a bounded wait on an asynchronous copy gave up
};

// finalize() operations
enum {
    FIN_F0 = 1,             // f0 = sum, resid = sqrt(f0)
    FIN_N3CUR = 2,          // n3max_cur = max
    FIN_AMAX = 4,           // n3max_next = max; alpha_max; weights for the first sample (or the fixed alpha)
    FIN_F1 = 8,             // f1 = sum; weights for the second sample
    FIN_F2_CHOOSE = 16,     // f2 = sum; alpha from the parabola; weights for the accepted point
    FIN_ACCEPT = 32,        // f0 = f3 = sum; n3max_cur = max; resid; iter++
    FIN_IDENTITY = 64,      // weights (1, 0) for a plain G evaluation
    FIN_F12_CHOOSE = 128    // f1 = sum, f2 = second sum (paired samples); alpha; weights for the accepted point
};
