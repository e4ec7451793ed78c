// Pass kernels of one residual evaluation G(rho) (Sec. "Discretization and Solution
// in Equilibrium"): every 3D transform is split into an x pass (rows, real <-> half
// spectrum), a y pass and a z pass (column tiles), and the pointwise work rides
// inside those passes:
//
//   first half  (rho -> weighted densities of eq. nDef, bulk-fluid + Poisson spectra)
//     k_xfwd     x R2C of the S densities
//     k_yfft     y forward
//     k_zconv_fwd  z forward, the analytic weights of App. B (n_hat_alpha), the
//                bulk-fluid kernel (eq. CplusPsiHat) and the Poisson symbol
//                (eq. potentialSolution) applied in k space, z inverse of the nine
//                weighted-density spectra (the x derivatives are formed in k_xphi)
//     k_yfft     y inverse of the nine spectra
//   second half (weighted densities -> c1 -> G)
//     k_xphi     x C2R to the ten n, dPhi/dn_alpha of eq. Phi (|nV2| <= n2 bound,
//                FP64 log(1-n3) and 1/(1-n3)^m; or another hard-sphere form), x R2C back
//                to nine spectra
//     k_yfft     y forward
//     k_zconv_bwd  z forward, adjoint weights (eq. muHS), + bulk-fluid/Poisson spectra,
//                z inverse of the S one-body correlations
//     k_yfft     y inverse
//     k_xupdate  x C2R and the update G_i = rho_bath_i exp(mu_HS_bath_i - V_i + c1_i)
//                (eq. rhoEquation), mixing of rho for the line search, residual sums
//
// Linear stages carry mixing weights (read from the device control block) so that
// n_alpha at a line-search point is the mix of two stored weighted-density sets:
// n3, and every n_alpha, is linear in rho (Sec. "Nonlinear solver").
#pragma once

#include <math_constants.h>

#include "common.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace dftk {

constexpr int kThreads = 256;
// the one-block line-search bookkeeping kernel: 1024 threads for many partial results, 256 for
// few (small grids, where its latency is all that counts)
constexpr int kFinThreads = 1024, kFinThreadsSmall = 256;


template <typename Real> __device__ __forceinline__ void sc(Real x, Real* s, Real* c);
template <> __device__ __forceinline__ void sc<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void sc<double>(double x, double* s, double* c) { sincos(x, s, c); }

// Wave number of index j on an axis of n points (eq. Kvalues); kf = 2 pi / (n h).
template <typename Real> __device__ __forceinline__ Real kval(int j, int n, Real kf) {
    return (2 * j <= n) ? Real(j) * kf : -Real(n - j) * kf;
}

// Power series sum_m (-1)^m y^(2m) / ((2m+1)! (2m+q)) in t = y^2, q = n + 3 of the ball
// integral (4 pi / k) I_n = 4 pi R^(n+3) * series (expansion of sin(k r) under the integral).
__host__ __device__ constexpr double series_coef(int m, int q) {
    double f = 1.0;
    for (int i = 2; i <= 2 * m + 1; ++i) f *= double(i);
    return ((m & 1) ? -1.0 : 1.0) / (f * double(2 * m + q));
}

template <typename Real, int Q> __device__ __forceinline__ Real ball_series(Real t) {
    constexpr int M = sizeof(Real) == 4 ? 9 : 11;
    Real acc = Real(0);
#pragma unroll
    for (int m = M - 1; m >= 0; --m) acc = acc * t + Real(series_coef(m, Q));
    return acc;
}

template <typename Real> __device__ __forceinline__ Real series_cut() { return sizeof(Real) == 4 ? Real(1.5) : Real(1.0); }

// (sin x - x cos x) / x^3 (1/3 at x = 0), s = sin x, c = cos x
template <typename Real> __device__ __forceinline__ Real sinc3(Real x, Real s, Real c) {
    if (x < series_cut<Real>()) return ball_series<Real, 3>(x * x);
    return (s - x * c) / (x * x * x);
}

// FMT scalar weights of App. B for one species at |k| (x = |k| R).  Returns w0 (w1 = R w0,
// w2 = 4 pi R^2 w0) and j3 = (sin x - x cos x)/x^3 (w3 = 4 pi R^3 j3).
template <typename Real> __device__ __forceinline__ void fmt_weights(Real kmag, Real R, Real* w0, Real* j3) {
    const Real x = kmag * R;
    Real s, c;
    sc<Real>(x, &s, &c);
    if (x < series_cut<Real>()) {
        // sin x / x series for accuracy next to the series of j3
        const Real t = x * x;
        *w0 = Real(1) + t * (Real(-1.0 / 6) + t * (Real(1.0 / 120) + t * (Real(-1.0 / 5040) + t * (Real(1.0 / 362880)
              + t * (Real(-1.0 / 39916800) + t * Real(1.0 / 6227020800.0))))));
    } else {
        *w0 = s / x;
    }
    *j3 = sinc3<Real>(x, s, c);
}

// Bulk-fluid kernel DC_ij_hat(|k|) of eq. CplusPsiHat (prefactor 2 pi lambda_B z_i z_j / k, i.e.
// (lambda_B z_i z_j / 2)(4 pi / k) I_n) in kT units.
template <typename Real>
__device__ __forceinline__ Real delta_c_hat(Real kmag, Real R, Real pref, Real a, Real b, Real c,
                                           Real* dGamma = nullptr, Real da = 0, Real db = 0, Real dc = 0) {
    const Real y = kmag * R;
    Real bm1, b0, b1;   // (4 pi / k) I_n / (4 pi R^(n+3))
    if (y < series_cut<Real>()) {
        const Real t = y * y;
        bm1 = ball_series<Real, 2>(t);
        b0 = ball_series<Real, 3>(t);
        b1 = ball_series<Real, 4>(t);
    } else {
        Real s, co;
        sc<Real>(y, &s, &co);
        Real sh, chh;
        sc<Real>(Real(0.5) * y, &sh, &chh);
        const Real omc = Real(2) * sh * sh;           // 1 - cos y, without cancellation
        const Real iy = Real(1) / y;
        const Real iy2 = iy * iy;
        bm1 = omc * iy2;
        b0 = (s - y * co) * iy2 * iy;
        b1 = -co * iy2 + Real(2) * s * iy2 * iy - Real(2) * omc * iy2 * iy2;
    }
    const Real R2 = R * R;
    const Real fourpi = Real(4.0 * CUDART_PI);
    // the Gamma dependence sits in the coefficients only (l_k = R_k + 1/(2 Gamma))
    if (dGamma) *dGamma = pref * fourpi * R2 * (da * R2 * b1 - db * R * b0 + dc * bm1);
    return pref * fourpi * R2 * (a * R2 * b1 - b * R * b0 + c * bm1);
}

// ------------------------------------------------------------------------------------
// Reductions
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < (int)(blockDim.x >> 5)) ? scratch[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

// Block sum of per-thread FP32 pairs (hi, lo) kept as a double-single (hi + lo) through the
// warp shuffles (error-free TwoSum of the high parts, Knuth), then in FP64 across the warps:
// about 48 significant bits at FP32 cost, where FP64 shuffles and adds would queue on the
// narrow FP64 pipe.  Result valid in thread 0.
__device__ __forceinline__ void ds_add(float& hi, float& lo, float bhi, float blo) {
    const float s = hi + bhi;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (bhi - bb);
    const float l = err + lo + blo;
    hi = s + l;
    lo = l - (hi - s);
}

__device__ __forceinline__ double block_sum_ds(float hi, float lo, double* scratch) {
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi, o), bl = __shfl_xor_sync(0xffffffffu, lo, o);
        ds_add(hi, lo, bh, bl);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = double(hi) + double(lo);
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += scratch[i];
    return r;
}

__device__ __forceinline__ float block_max(float v, float* scratch) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    float r = -CUDART_INF_F;
    if (threadIdx.x < 32) {
        r = (l < (int)(blockDim.x >> 5)) ? scratch[l] : -CUDART_INF_F;
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    return r;
}

// Position of element e within an x-pass row: padded in the compile-time passes (see ct_xpad).
template <int NX> __device__ __forceinline__ int xo(int e) { return NX > 0 ? ct_xpad(e) : e; }

template <typename C> __device__ __forceinline__ C* align_ptr(unsigned char* p) {
    uintptr_t u = reinterpret_cast<uintptr_t>(p);
    u = (u + 15) & ~uintptr_t(15);
    return reinterpret_cast<C*>(u);
}

// Copy a column tile (n rows of T complex, global row stride rs, columns t < valid) between
// global and shared memory ([e][t] layout).  TT/NN > 0: compile-time tile, loads batched in
// registers so that all of a thread's loads are in flight together.
template <int TT, int NN, typename C>
__device__ __forceinline__ void tile_load(C* __restrict__ dst, const C* __restrict__ src, long long rs, int valid,
                                          int T, int n) {
    if constexpr (TT > 0 && NN > 0) {
        constexpr int TOTAL = TT * NN;
        constexpr int PER = (TOTAL + kThreads - 1) / kThreads;
        C tmp[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            const int e = idx / TT, t = idx % TT;
            tmp[i] = cmake<C>(0, 0);
            if ((TOTAL % kThreads == 0 || idx < TOTAL) && t < valid) tmp[i] = src[e * rs + t];
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            if (TOTAL % kThreads == 0 || idx < TOTAL) dst[idx] = tmp[i];
        }
    } else {
        for (int idx = threadIdx.x; idx < T * n; idx += blockDim.x) {
            const int e = idx / T, t = idx - (idx / T) * T;
            dst[idx] = (t < valid) ? src[e * rs + t] : cmake<C>(0, 0);
        }
    }
}

template <int TT, int NN, typename C>
__device__ __forceinline__ void tile_store(C* __restrict__ dst, const C* __restrict__ src, long long rs, int valid,
                                           int T, int n) {
    if constexpr (TT > 0 && NN > 0) {
        constexpr int TOTAL = TT * NN;
#pragma unroll
        for (int idx = threadIdx.x; idx < TOTAL; idx += kThreads) {
            const int e = idx / TT, t = idx % TT;
            if (t < valid) dst[e * rs + t] = src[idx];
        }
    } else {
        for (int idx = threadIdx.x; idx < T * n; idx += blockDim.x) {
            const int e = idx / T, t = idx - (idx / T) * T;
            if (t < valid) dst[e * rs + t] = src[idx];
        }
    }
}

// ------------------------------------------------------------------------------------
// x pass, forward: S real fields -> half spectra.  Two real rows a, b are packed as a + i b
// into one complex transform of length nx and separated afterwards:
//   X_a[k] = (Z[k] + conj Z[-k]) / 2,  X_b[k] = (Z[k] - conj Z[-k]) / (2 i).
// ------------------------------------------------------------------------------------
template <typename Real, int NX>
__global__ void __launch_bounds__(kThreads) k_xfwd(GridDesc g, AxisPlan px, int ncomp, int lx,
                                                   const Real* __restrict__ in,
                                                   typename Cplx<Real>::type* __restrict__ out,
                                                   const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lx * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long rows = (long long)ncomp * g.ny * g.nz;
    const long long pair0 = (long long)blockIdx.x * lx;
    // rows 2(pair0 + l) and 2(pair0 + l) + 1 as the real and imaginary parts of line l; the loads
    // of kU elements per thread are issued before their shared-memory stores
    constexpr int kU = 4;
    const int total = lx * nx;
    for (int base = threadIdx.x; base < total; base += kU * kThreads) {
        Real av[kU], bv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = base + u * kThreads;
            const int l = idx / nx, x = idx - (idx / nx) * nx;
            const long long ra = 2 * (pair0 + l), rb = ra + 1;
            av[u] = (idx < total && ra < rows) ? in[ra * nx + x] : Real(0);
            bv[u] = (idx < total && rb < rows) ? in[rb * nx + x] : Real(0);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = base + u * kThreads;
            if (idx >= total) break;
            const int l = idx / nx, x = idx - (idx / nx) * nx;
            A[l * pitch + xo<NX>(x)] = cmake<C>(av[u], bv[u]);
        }
    }
    __syncthreads();
    C* R = any_fft<NX, false, false, 0>(A, B, px, lx, 1, pitch, tw);
    for (int idx = threadIdx.x; idx < lx * nxh; idx += blockDim.x) {
        const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
        const long long ra = 2 * (pair0 + l), rb = ra + 1;
        const C zk = R[l * pitch + xo<NX>(k)];
        const C znk = R[l * pitch + xo<NX>(k == 0 ? 0 : nx - k)];
        const C s = cadd(zk, cconj(znk));
        const C d = csub(zk, cconj(znk));
        if (ra < rows) out[ra * g.pxh + k] = cmake<C>(Real(0.5) * s.x, Real(0.5) * s.y);
        if (rb < rows) out[rb * g.pxh + k] = cmake<C>(Real(0.5) * d.y, Real(-0.5) * d.x);
    }
}

// ------------------------------------------------------------------------------------
// y pass: in-place transform of ncomp half spectra along y, tiles of T kx columns.
// grid (ceil(nxh/T), nz, ncomp)
// ------------------------------------------------------------------------------------
template <typename Real, bool INV, int NY, int TY>
__global__ void __launch_bounds__(kThreads) k_yfft(GridDesc g, AxisPlan py, int Trt,
                                                   typename Cplx<Real>::type* __restrict__ data,
                                                   const typename Cplx<Real>::type* __restrict__ twy) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    const int ny = NY > 0 ? NY : g.ny, nxh = g.nxh, pxh = g.pxh;
    const int T = TY > 0 ? TY : Trt;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + ny;
    C* B = A + T * ny;
    for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = twy[i];
    const int kx0 = blockIdx.x * T;
    C* base = data + (long long)blockIdx.z * g.nc + (long long)blockIdx.y * ny * pxh + kx0;
    tile_load<TY, NY>(A, base, pxh, nxh - kx0, T, ny);
    __syncthreads();
    C* R = any_fft<NY, INV, true, TY>(A, B, py, T, T, 1, tw);
    tile_store<TY, NY>(base, R, pxh, nxh - kx0, T, ny);
}

// ------------------------------------------------------------------------------------
// y pass with TMA tiles (compile-time length NY <= 256 and tile width TY).  Persistent: CTA b
// handles tiles b, b + gridDim.x, ...  Two shared-memory stages are filled by TMA loads (one
// cp.async.bulk.tensor per tile, completing on an mbarrier).  The first FFT stage moves a
// tile out of its TMA stage into scratch X, so the stage is refilled with the tile after next
// at once; the remaining stages run between X and Y (padded layout) and the last writes the
// dense box that leaves through a TMA store, whose shared-memory reads are awaited only before
// that buffer is written again.  The tensor map views the half spectra as (x: nxh * E, y: ny,
// plane: nz * ncomp) 8-byte elements, E = sizeof(complex) / 8; a tile is the box (TY * E, NY,
// 1).  A wait that runs out sets DEV_TIMEOUT and the CTA stops after draining the loads it has
// in flight.
// Shared memory: stage 0 | stage 1 (dense tiles) | X | Y (padded) | twiddles | 2 mbarriers.
// ------------------------------------------------------------------------------------
template <typename Real, int NY, int TY> __host__ __device__ constexpr size_t yfft_tma_smem() {
    using C = typename Cplx<Real>::type;
    return (2 * size_t(TY) * NY + 2 * size_t(ct_gstride(NY, TY, int(sizeof(C)))) + NY) * sizeof(C) +
           2 * sizeof(uint64_t) + 128;
}

// ZAX: the same pass along z.  The map is then the z passes' view (x: nxh * E, y: ny, plane:
// nz * ncomp) with box (TY * E, 1, NY): a tile is TY kx columns of all NY z points at one ky
// of one component, tile t = (kx tile, ky + ny c) -> coordinates (x, ky, c NY); the box lands in
// shared memory with the same layout (element (z, t) at z TY + t) as a y tile's.
template <typename Real, bool INV, int NY, int TY, bool ZAX = false>
__global__ void __launch_bounds__(kThreads) k_yfft_tma(const __grid_constant__ CUtensorMap map, int ntiles_x,
                                                       int ntiles, int* __restrict__ status,
                                                       const typename Cplx<Real>::type* __restrict__ twy,
                                                       long long polls, int ny_planes = 1) {
    dep_launch();
    dep_wait();
    static_assert(NY > 0 && NY <= 256 && TY > 0, "compile-time TMA y pass");
    using C = typename Cplx<Real>::type;
    constexpr int E = int(sizeof(C) / 8);
    constexpr int TILE = TY * NY;
    constexpr int GS = ct_gstride(NY, TY, int(sizeof(C)));
    constexpr int NST = ct_nstages(NY);
    constexpr uint32_t BYTES = uint32_t(TILE * sizeof(C));
    static_assert(BYTES % 128 == 0, "TMA stage alignment");
    extern __shared__ unsigned char smem_raw[];
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127);
    C* const stage0 = reinterpret_cast<C*>(base);
    C* X = stage0 + 2 * TILE;
    C* Y = X + GS;
    C* tw = Y + GS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + NY);
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < NY; i += kThreads) tw[i] = twy[i];
    __syncthreads();
    // tensor-map coordinates of a tile
    auto cy = [&](int tile) { return ZAX ? (tile / ntiles_x) % ny_planes : 0; };
    auto cz = [&](int tile) { return ZAX ? (tile / ntiles_x) / ny_planes * NY : tile / ntiles_x; };
    int issued = 0, consumed = 0;   // per stage, packed (stage 1 << 16) | stage 0; thread 0
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            const int tile = blockIdx.x + s * gridDim.x;
            if (tile < ntiles) {
                tma::mbar_expect_tx(&bar[s], BYTES);
                tma::load_3d(stage0 + s * TILE, &map, (tile % ntiles_x) * TY * E, cy(tile), cz(tile), &bar[s]);
                issued += 1 << (16 * s);
            }
        }
    }
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int cur = it & 1;
        C* st = stage0 + cur * TILE;
        const bool ok = tma::mbar_wait(&bar[cur], (it >> 1) & 1, polls);
        // an odd stage count leaves the result in X, which the first stage writes next
        if (NST % 2 == 1 && threadIdx.x == 0) tma::wait_read_all();
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, DEV_TIMEOUT);
                for (int s = 0; s < 2; ++s) {
                    const int n_is = (issued >> (16 * s)) & 0xffff, n_co = (consumed >> (16 * s)) & 0xffff;
                    if (n_is > n_co) tma::mbar_wait(&bar[s], (n_is - 1) & 1);
                }
            }
            break;
        }
        consumed += 1 << (16 * cur);
        ct_stage_grouped<NY, ct_radix_at(NY, 0), ct_ns_at(NY, 0), INV, TY, GS, true, NST == 1, kThreads>(st, X, 1,
                                                                                                       tw);
        // an even stage count leaves the result in Y, which the second stage writes next
        if (NST % 2 == 0 && threadIdx.x == 0) tma::wait_read_all();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int next = tile + 2 * gridDim.x;
            if (next < ntiles) {
                tma::mbar_expect_tx(&bar[cur], BYTES);
                tma::load_3d(st, &map, (next % ntiles_x) * TY * E, cy(next), cz(next), &bar[cur]);
                issued += 1 << (16 * cur);
            }
        }
        C* a = X;
        C* b = Y;
        ct_stages_grouped<NY, INV, TY, GS, false, true, kThreads, 1>(a, b, 1, tw);
        tma::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma::store_3d(&map, (tile % ntiles_x) * TY * E, cy(tile), cz(tile), a);
            tma::commit();
        }
    }
    if (threadIdx.x == 0) tma::wait_all();
}

// Wave vector components of tile point (kz index, t) in a z-pass tile at (kx0, ky index)
template <typename Real> struct KPoint {
    Real kx, ky, kz, kmag;
    bool nyq_x, nyq_y, nyq_z, zero;
};

template <typename Real>
__device__ __forceinline__ KPoint<Real> kpoint(const GridDesc& g, int kxi, int kyi, int kzi, Real kfx, Real kfy,
                                               Real kfz) {
    KPoint<Real> p;
    p.kx = kval<Real>(kxi, g.nx, kfx);
    p.ky = kval<Real>(kyi, g.ny, kfy);
    p.kz = kval<Real>(kzi, g.nz, kfz);
    p.kmag = sqrt(p.kx * p.kx + p.ky * p.ky + p.kz * p.kz);
    p.nyq_x = (g.nx % 2 == 0) && (2 * kxi == g.nx);
    p.nyq_y = (g.ny % 2 == 0) && (2 * kyi == g.ny);
    p.nyq_z = (g.nz % 2 == 0) && (2 * kzi == g.nz);
    p.zero = (kxi == 0) && (kyi == 0) && (kzi == 0);
    return p;
}

// Bulk-fluid + mean-field kernel K_ij(k) = DC_ij_hat(k) - 4 pi lambda_B z_i z_j / lap(k) (k != 0),
// lap(k) = sum_d 4 sin^2(k_d h_d / 2) / h_d^2 (eq. potentialSolution), psi_hat(0) = 0.
template <typename Real>
__device__ __forceinline__ Real es_kernel(const SpeciesDesc<Real>& sp, int i, int j, const KPoint<Real>& p, Real inv_lap,
                                         Real* dGamma = nullptr) {
    Real K = delta_c_hat<Real>(p.kmag, sp.es_R[i][j], sp.es_pref[i][j], sp.es_a[i][j], sp.es_b[i][j], sp.es_c[i][j],
                               dGamma, sp.es_da[i][j], sp.es_db[i][j], sp.es_dc[i][j]);
    if (!p.zero) K -= sp.pois[i][j] * inv_lap;
    return K;
}

// One axis's term of lap(k): sin^2(k_d h_d / 2) / h_d^2.
template <typename Real> __device__ __forceinline__ Real lap_term(Real k, Real h) {
    const Real s = sin(Real(0.5) * k * h);
    return s * s / (h * h);
}

template <typename Real>
__device__ __forceinline__ Real inverse_laplacian(const KPoint<Real>& p, Real hx, Real hy, Real hz) {
    if (p.zero) return Real(0);
    const Real lap = Real(4) * (lap_term(p.kx, hx) + lap_term(p.ky, hy) + lap_term(p.kz, hz));
    return Real(1) / lap;
}

// The same from the plan's per-axis table (sp.lap1d, the lap_term values by FFT index, evaluated
// by k_laptab with the same expression: equal bit for bit) where it has one.
template <typename Real>
__device__ __forceinline__ Real inverse_laplacian(const SpeciesDesc<Real>& sp, const GridDesc& g, const KPoint<Real>& p,
                                                  int kxi, int kyi, int kzi, Real hx, Real hy, Real hz) {
    if (!sp.lap1d) return inverse_laplacian<Real>(p, hx, hy, hz);
    if (p.zero) return Real(0);
    const Real lap = Real(4) * (__ldg(sp.lap1d + kxi) + __ldg(sp.lap1d + g.nx + kyi) + __ldg(sp.lap1d + g.nx + g.ny + kzi));
    return Real(1) / lap;
}

// The per-axis Laplacian terms of a grid: out[i] for x indices i < nx, out[nx + j] for y, out[nx +
// ny + l] for z (wave numbers kval of the FFT index, as the z passes form them).
template <typename Real>
__global__ void k_laptab(GridDesc g, Real kfx, Real kfy, Real kfz, Real* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx + g.ny + g.nz) return;
    Real v;
    if (i < g.nx) v = lap_term(kval<Real>(i, g.nx, kfx), Real(g.hx));
    else if (i < g.nx + g.ny) v = lap_term(kval<Real>(i - g.nx, g.ny, kfy), Real(g.hy));
    else v = lap_term(kval<Real>(i - g.nx - g.ny, g.nz, kfz), Real(g.hz));
    out[i] = v;
}

// ------------------------------------------------------------------------------------
// z pass of the first half.  grid (ceil(nxh/T), ny)
//   in:      S half spectra after x, y forward  (kx, ky, z)
//   slot_n:  10 weighted densities, 1/N applied, after z inverse (kx, ky, z)
//   slot_es: S (+1 with psi) unnormalised bulk-fluid/Poisson spectra sum_j K_ij drho_hat_j (kx, ky, kz)
// Shared pool of 7 tiles of T x nz.
// ------------------------------------------------------------------------------------
template <typename Real, int NZ, int TZ, bool GRAD>
__global__ void __launch_bounds__(kThreads) k_zconv_fwd(GridDesc g, AxisPlan pz, SpeciesDesc<Real> sp, int Trt,
                                                        Real kfx, Real kfy, Real kfz, int want_psi,
                                                        const typename Cplx<Real>::type* __restrict__ in,
                                                        typename Cplx<Real>::type* __restrict__ slot_n,
                                                        typename Cplx<Real>::type* __restrict__ slot_es,
                                                        double* __restrict__ red_energy,
                                                        const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double scratch_d[32];
    const int nz = NZ > 0 ? NZ : g.nz, ny = g.ny, nxh = g.nxh, S = sp.S;
    // red_energy (optional): per block, [0] = sum_k w Re(conj(drho_hat_i) es_hat_i) and
    // [1] = sum_k w Re(conj(drho_hat_i) dK_ij/dGamma drho_hat_j), w = 1 on the kx = 0 and Nyquist
    // planes and 2 elsewhere (the half spectrum standing for the full one)
    double e_acc = 0.0, q_acc = 0.0;
    const int T = TZ > 0 ? TZ : Trt;
    const int tile = T * nz;
    C* tw = align_ptr<C>(smem_raw);
    C* pool[7];
    for (int i = 0; i < 7; ++i) pool[i] = tw + nz + i * tile;
    for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = twz[i];
    const int kx0 = blockIdx.x * T;
    const int kyi = blockIdx.y;
    const long long zstride = (long long)ny * g.pxh;
    const long long col0 = (long long)kyi * g.pxh + kx0;

    // phase 1: forward z transform of each species tile; results end in pool[0..S-1]
    for (int s = 0; s < S; ++s) {
        C* b = pool[s];
        tile_load<TZ, NZ>(b, in + (long long)s * g.nc + col0, zstride, nxh - kx0, T, nz);
        __syncthreads();
        C* r = any_fft<NZ, false, true, TZ>(b, pool[6], pz, T, T, 1, tw);
        if (r != b) { pool[6] = b; pool[s] = r; }
    }

    // phase 2: k-space products at each tile point
    const Real hx = Real(g.hx), hy = Real(g.hy), hz = Real(g.hz);
    const Real fourpi = Real(4.0 * CUDART_PI);
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int kzi = idx / T, t = idx - (idx / T) * T;
        const int kxi = kx0 + t;
        const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
        C v[DFT_MAXS];
        for (int s = 0; s < S; ++s) v[s] = pool[s][idx];
        C acc[5];
        for (int a = 0; a < 5; ++a) acc[a] = cmake<C>(Real(0), Real(0));
        for (int s = 0; s < S; ++s) {
            Real w0, j3;
            fmt_weights<Real>(p.kmag, sp.R[s], &w0, &j3);
            const Real R = sp.R[s];
            acc[0] = cadd(acc[0], cscale(v[s], w0));
            acc[1] = cadd(acc[1], cscale(v[s], R * w0));
            acc[2] = cadd(acc[2], cscale(v[s], fourpi * R * R * w0));
            acc[3] = cadd(acc[3], cscale(v[s], fourpi * R * R * R * j3));
            acc[4] = cadd(acc[4], cscale(v[s], R * R * j3));       // w3 / (4 pi R)
        }
        if (kxi < nxh) {
            const Real inv_lap = inverse_laplacian<Real>(sp, g, p, kxi, kyi, kzi, hx, hy, hz);
            C dv[DFT_MAXS];
            for (int s = 0; s < S; ++s) {
                dv[s] = v[s];
                if (p.zero) dv[s].x -= sp.n_rho_b[s];       // DFT(rho - rho_bath) at k = 0
            }
            C es[DFT_MAXS];
            for (int s = 0; s < S; ++s) es[s] = cmake<C>(Real(0), Real(0));
            const double wk = GRAD ? ((kxi == 0 || (g.nx % 2 == 0 && 2 * kxi == g.nx)) ? 1.0 : 2.0) : 0.0;
            for (int i = 0; i < S; ++i) {
                for (int j = i; j < S; ++j) {
                    Real dK = Real(0);
                    const Real K = es_kernel<Real>(sp, i, j, p, inv_lap, GRAD ? &dK : nullptr);
                    es[i] = cadd(es[i], cscale(dv[j], K));
                    if (j != i) es[j] = cadd(es[j], cscale(dv[i], K));
                    if constexpr (GRAD) {
                        const double re = double(dv[i].x) * dv[j].x + double(dv[i].y) * dv[j].y;
                        q_acc += wk * double(dK) * re * (j != i ? 2.0 : 1.0);
                    }
                }
            }
            if constexpr (GRAD)
                for (int i = 0; i < S; ++i) e_acc += wk * (double(dv[i].x) * es[i].x + double(dv[i].y) * es[i].y);
            const long long o = (long long)kzi * zstride + col0 + t;
            for (int s = 0; s < S; ++s) slot_es[(long long)s * g.nc + o] = es[s];
            if (want_psi) {
                C q = cmake<C>(Real(0), Real(0));
                for (int s = 0; s < S; ++s) q = cadd(q, cscale(v[s], sp.z[s]));
                // psi_hat = 4 pi lambda_B q_hat / lap; pois[s][s] / z_s^2 = 4 pi lambda_B
                Real flb = Real(0);
                for (int s = 0; s < S; ++s)
                    if (sp.z[s] != Real(0)) { flb = sp.pois[s][s] / (sp.z[s] * sp.z[s]); break; }
                slot_es[(long long)S * g.nc + o] = cscale(q, flb * inv_lap);
            }
        }
        for (int a = 0; a < 5; ++a) pool[a][idx] = cscale(acc[a], sp.inv_n);
    }
    if constexpr (GRAD) {
        const double be = block_sum(e_acc, scratch_d);
        const double bq = block_sum(q_acc, scratch_d);
        if (threadIdx.x == 0) {
            const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            red_energy[2 * b] = be;
            red_energy[2 * b + 1] = bq;
        }
    }
    __syncthreads();

    // phase 3: inverse z of the nine weighted-density spectra: n0..n3, m, then i k_y m, i k_z m,
    // i k_y n3, i k_z n3 (zero on the Nyquist index of their axis); the derived ones first,
    // while m and n3 are still in k space.
    const int order[DFT_NSPEC] = {5, 6, 7, 8, 4, 3, 0, 1, 2};
    for (int oi = 0; oi < DFT_NSPEC; ++oi) {
        const int a = order[oi];
        C* r;
        if (a >= 5) {
            const C* src = (a < 7) ? pool[4] : pool[3];
            const int d = (a == 5 || a == 7) ? 1 : 2;
            C* W = pool[5];
            for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
                const int kzi = idx / T;
                Real kd;
                bool nyq;
                if (d == 1) { kd = kval<Real>(kyi, g.ny, kfy); nyq = (g.ny % 2 == 0) && (2 * kyi == g.ny); }
                else { kd = kval<Real>(kzi, g.nz, kfz); nyq = (g.nz % 2 == 0) && (2 * kzi == g.nz); }
                const C u = src[idx];
                W[idx] = nyq ? cmake<C>(Real(0), Real(0)) : cmake<C>(-kd * u.y, kd * u.x);
            }
            __syncthreads();
            r = any_fft<NZ, true, true, TZ>(W, pool[6], pz, T, T, 1, tw);
        } else {
            r = any_fft<NZ, true, true, TZ>(pool[a], pool[5], pz, T, T, 1, tw);
        }
        tile_store<TZ, NZ>(slot_n + (long long)a * g.nc + col0, r, zstride, nxh - kx0, T, nz);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Grouped z passes (compile-time length NZ, tile width TZ), grid (ceil(nxh/TZ), ny).  All
// components of a column tile are loaded in one batch of in-flight loads and transformed by
// one grouped FFT (ct_fft_grouped), so every stage keeps the CTA's threads busy and a tile
// costs a handful of barriers instead of a dozen transforms of one component each.
// Shared memory: twiddles | 10 tiles | 10 tiles (ct_gstride(NZ, TZ, csize) elements each).
// ------------------------------------------------------------------------------------
// The nine weighted-density spectra of one k point into grouped tiles (group stride GS,
// position pos), 1/N applied: acc = (n0, n1, n2, n3, m) spectra; i k_y and i k_z of m and n3
// are zero on the Nyquist index of their axis.
template <typename Real>
__device__ __forceinline__ void store_wd_spectra(typename Cplx<Real>::type* O, int GS, int pos,
                                                 const typename Cplx<Real>::type* acc, Real inv_n,
                                                 const KPoint<Real>& p) {
    using C = typename Cplx<Real>::type;
#pragma unroll
    for (int a = 0; a < 5; ++a) O[a * GS + pos] = cscale(acc[a], inv_n);
    const C m = cscale(acc[4], inv_n), n3 = cscale(acc[3], inv_n);
    const C zero = cmake<C>(Real(0), Real(0));
    O[5 * GS + pos] = p.nyq_y ? zero : cmake<C>(-p.ky * m.y, p.ky * m.x);
    O[6 * GS + pos] = p.nyq_z ? zero : cmake<C>(-p.kz * m.y, p.kz * m.x);
    O[7 * GS + pos] = p.nyq_y ? zero : cmake<C>(-p.ky * n3.y, p.ky * n3.x);
    O[8 * GS + pos] = p.nyq_z ? zero : cmake<C>(-p.kz * n3.y, p.kz * n3.x);
}

// Species-independent sums of the back convolution at one k point from the nine Phi' spectra
// of the x and y passes (group stride GS, position pos): a0..a2 = Phi_0..Phi_2,
// a3 = B3 - i k_y Phi_V2y - i k_z Phi_V2z, a4 = B4 - i k_y Phi_V1y - i k_z Phi_V1z, where the
// x pass formed B3 = Phi_3 - i k_x Phi_V2x and B4 = -i k_x Phi_V1x (Nyquist terms dropped).
template <typename Real>
__device__ __forceinline__ void bwd_sums(const typename Cplx<Real>::type* X, int GS, int pos, const KPoint<Real>& p,
                                         typename Cplx<Real>::type* a) {
    using C = typename Cplx<Real>::type;
    a[0] = X[0 * GS + pos];
    a[1] = X[1 * GS + pos];
    a[2] = X[2 * GS + pos];
    a[3] = X[3 * GS + pos];
    a[4] = X[4 * GS + pos];
    if (!p.nyq_y) {
        const C u1 = X[5 * GS + pos], u2 = X[7 * GS + pos];
        a[4] = cadd(a[4], cmake<C>(p.ky * u1.y, -p.ky * u1.x));
        a[3] = cadd(a[3], cmake<C>(p.ky * u2.y, -p.ky * u2.x));
    }
    if (!p.nyq_z) {
        const C u1 = X[6 * GS + pos], u2 = X[8 * GS + pos];
        a[4] = cadd(a[4], cmake<C>(p.kz * u1.y, -p.kz * u1.x));
        a[3] = cadd(a[3], cmake<C>(p.kz * u2.y, -p.kz * u2.x));
    }
}

// The persistent TMA z passes transform seven of the nine spectra: the y-derivative spectra
// (components 5 and 7: i k_y m and i k_y n3, or their Phi' counterparts) differ from the m and n3
// spectra by the factor i k_y, which is one constant per z tile, so it is applied on the tile
// (after the first half's z inverse, before the second half's z forward) instead of transforming
// them.  In a tile's shared memory, component c sits at group zgroup(c): the seven transformed
// spectra first (0..4, then i k_z m, i k_z n3), the two y-derivative spectra at 7 and 8 (the
// fold partners of groups 4 and 3).
constexpr int kZGroups = 7;
__host__ __device__ constexpr int zgroup(int c) { return c < 5 ? c : (c == 5 ? 7 : c == 6 ? 5 : c == 7 ? 8 : 6); }

// bwd_sums on the seven transformed groups, the y derivatives already folded into groups 3 and 4
// (a3 = B3 - i k_y Phi_V2y, a4 = B4 - i k_y Phi_V1y): the z derivatives remain.
template <typename Real>
__device__ __forceinline__ void bwd_sums_folded(const typename Cplx<Real>::type* X, int GS, int pos,
                                                const KPoint<Real>& p, typename Cplx<Real>::type* a) {
    using C = typename Cplx<Real>::type;
#pragma unroll
    for (int q = 0; q < 5; ++q) a[q] = X[q * GS + pos];
    if (!p.nyq_z) {
        const C u1 = X[zgroup(6) * GS + pos], u2 = X[zgroup(8) * GS + pos];
        a[4] = cadd(a[4], cmake<C>(p.kz * u1.y, -p.kz * u1.x));
        a[3] = cadd(a[3], cmake<C>(p.kz * u2.y, -p.kz * u2.x));
    }
}

// store_wd_spectra without the y derivatives: groups 0..4 and i k_z m, i k_z n3 at zgroup(6),
// zgroup(8); the z inverse transforms these seven and zfwd_add_y_derivatives forms the other two.
template <typename Real>
__device__ __forceinline__ void store_wd_spectra_z(typename Cplx<Real>::type* O, int GS, int pos,
                                                   const typename Cplx<Real>::type* acc, Real inv_n,
                                                   const KPoint<Real>& p) {
    using C = typename Cplx<Real>::type;
#pragma unroll
    for (int a = 0; a < 5; ++a) O[a * GS + pos] = cscale(acc[a], inv_n);
    const C m = cscale(acc[4], inv_n), n3 = cscale(acc[3], inv_n);
    const C zero = cmake<C>(Real(0), Real(0));
    O[zgroup(6) * GS + pos] = p.nyq_z ? zero : cmake<C>(-p.kz * m.y, p.kz * m.x);
    O[zgroup(8) * GS + pos] = p.nyq_z ? zero : cmake<C>(-p.kz * n3.y, p.kz * n3.x);
}

// After the first half's z inverse (dense tiles, TILE elements per group): the y-derivative
// spectra i k_y m -> zgroup(5), i k_y n3 -> zgroup(7), zero on the Nyquist index of y.
template <typename Real, int TILE, int NT>
__device__ __forceinline__ void zfwd_add_y_derivatives(typename Cplx<Real>::type* Q, int GS, Real ky) {
    using C = typename Cplx<Real>::type;
    for (int idx = threadIdx.x; idx < 2 * TILE; idx += NT) {
        const int h = idx / TILE, e = idx - h * TILE;
        const C u = Q[(h ? 3 : 4) * GS + e];
        Q[(h ? zgroup(7) : zgroup(5)) * GS + e] = cmake<C>(-ky * u.y, ky * u.x);
    }
}

template <int TT, int NN> __host__ __device__ constexpr size_t zg_smem_bytes(size_t csize) {
    return (size_t(NN) + 2 * size_t(DFT_NSPEC) * ct_gstride(NN, TT, int(csize))) * csize + 16;
}

// Load `groups` column tiles (component c at src + c * cstride, global row stride rs, columns
// t < valid, zero elsewhere) into the grouped layout; every load of a thread is issued before
// its first shared-memory store.
template <int TT, int NN, int GMAX, typename C>
__device__ __forceinline__ void tiles_load_grouped(C* __restrict__ dst, const C* __restrict__ src, long long cstride,
                                                   int groups, long long rs, int valid) {
    constexpr int TILE = TT * NN;
    constexpr int PER = (TILE + kThreads - 1) / kThreads;
    constexpr int GS = ct_gstride(NN, TT, int(sizeof(C)));
    C reg[GMAX][PER];
#pragma unroll
    for (int gi = 0; gi < GMAX; ++gi) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            const int e = idx / TT, t = idx % TT;
            reg[gi][i] = cmake<C>(0, 0);
            if (gi < groups && (TILE % kThreads == 0 || idx < TILE) && t < valid)
                reg[gi][i] = src[gi * cstride + e * rs + t];
        }
    }
#pragma unroll
    for (int gi = 0; gi < GMAX; ++gi) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            const int e = idx / TT, t = idx % TT;
            if (gi < groups && (TILE % kThreads == 0 || idx < TILE)) dst[gi * GS + ct_gpos(e, TT) + t] = reg[gi][i];
        }
    }
}

template <int TT, int NN, typename C>
__device__ __forceinline__ void tiles_store_grouped(C* __restrict__ dst, const C* __restrict__ src, long long cstride,
                                                    int groups, long long rs, int valid) {
    constexpr int TILE = TT * NN;
    constexpr int GS = ct_gstride(NN, TT, int(sizeof(C)));
    for (int gi = 0; gi < groups; ++gi) {
#pragma unroll
        for (int idx = threadIdx.x; idx < TILE; idx += kThreads) {
            const int e = idx / TT, t = idx % TT;
            if (t < valid) dst[gi * cstride + e * rs + t] = src[gi * GS + ct_gpos(e, TT) + t];
        }
    }
}

// Load the first n entries of a table record (16-byte aligned) with 16-byte loads.
template <typename Real, int MAXN>
__device__ __forceinline__ void load_record(Real (&dst)[MAXN], const Real* __restrict__ rec, int n) {
    constexpr int V = int(16 / sizeof(Real));
    static_assert(MAXN % V == 0, "record capacity");
#pragma unroll
    for (int v = 0; v < MAXN / V; ++v) {
        if (v * V < n) {
            if constexpr (sizeof(Real) == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4*>(rec) + v);
                dst[4 * v] = t.x; dst[4 * v + 1] = t.y; dst[4 * v + 2] = t.z; dst[4 * v + 3] = t.w;
            } else {
                const double2 t = __ldg(reinterpret_cast<const double2*>(rec) + v);
                dst[2 * v] = t.x; dst[2 * v + 1] = t.y;
            }
        }
    }
}

// Tables of the |k|-only factors for a cubic box (kf equal on the three axes): the FMT weights
// w0, j3 of each species and the bulk-fluid kernel DC_ij_hat with its Gamma derivative, at
// |k| = kf sqrt(m2) for every integer m2 in [0, m2max].  Evaluated once per plan with the same
// functions the z passes call per point.
template <typename Real>
__global__ void k_ktab(SpeciesDesc<Real> sp, double kf, int m2max, Real* tab_w, Real* tab_k, Real* tab_dk) {
    const int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (m2 > m2max) return;
    const int S = sp.S;
    const Real kmag = Real(kf * sqrt(double(m2)));
    for (int s = 0; s < S; ++s) {
        Real w0, j3;
        fmt_weights<Real>(kmag, sp.R[s], &w0, &j3);
        tab_w[(long long)m2 * sp.tab_ws + 2 * s] = w0;
        tab_w[(long long)m2 * sp.tab_ws + 2 * s + 1] = j3;
    }
    for (int j = 0; j < S; ++j)
        for (int i = 0; i <= j; ++i) {
            Real dG = Real(0);
            const Real K = delta_c_hat<Real>(kmag, sp.es_R[i][j], sp.es_pref[i][j], sp.es_a[i][j], sp.es_b[i][j],
                                             sp.es_c[i][j], &dG, sp.es_da[i][j], sp.es_db[i][j], sp.es_dc[i][j]);
            tab_k[(long long)m2 * sp.tab_ks + dft_pair(i, j)] = K;
            tab_dk[(long long)m2 * sp.tab_ks + dft_pair(i, j)] = dG;
        }
}

__device__ __forceinline__ int signed_index(int j, int n) { return (2 * j <= n) ? j : j - n; }
// m^2 = mx^2 + my^2 + mz^2 of a cubic box's mode (the |k| table index) from kx index kxi >= 0,
// signed y index my and z index kzi
__device__ __forceinline__ int kmode2(int kxi, int my, int kzi, int nz) {
    const int mz = signed_index(kzi, nz);
    return kxi * kxi + my * my + mz * mz;
}

// First-half z pass (same contract as k_zconv_fwd): S species spectra in, the ten weighted
// densities (z inverse, 1/N applied) and the bulk-fluid/Poisson spectra out.  Per-species loops
// run to DFT_MAXS with guards so that every per-point array stays in registers.
template <typename Real, int NZ, int TZ, bool GRAD>
__global__ void __launch_bounds__(kThreads, 2) k_zconv_fwd_g(GridDesc g, SpeciesDesc<Real> sp, Real kfx, Real kfy,
                                                             Real kfz, int want_psi,
                                                             const typename Cplx<Real>::type* __restrict__ in,
                                                             typename Cplx<Real>::type* __restrict__ slot_n,
                                                             typename Cplx<Real>::type* __restrict__ slot_es,
                                                             double* __restrict__ red_energy,
                                                             const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    constexpr int TILE = TZ * NZ;
    constexpr int GS = ct_gstride(NZ, TZ, int(sizeof(C)));
    extern __shared__ unsigned char smem_raw[];
    __shared__ double scratch_d[32];
    const int ny = g.ny, nxh = g.nxh, S = sp.S;
    const int Pn = S * (S + 1) / 2;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + NZ;
    C* B = A + DFT_NSPEC * GS;
    for (int i = threadIdx.x; i < NZ; i += kThreads) tw[i] = twz[i];
    const int kx0 = blockIdx.x * TZ;
    const int kyi = blockIdx.y;
    const long long zstride = (long long)ny * g.pxh;
    const long long col0 = (long long)kyi * g.pxh + kx0;
    tiles_load_grouped<TZ, NZ, DFT_MAXS>(A, in + col0, g.nc, S, zstride, nxh - kx0);
    __syncthreads();
    C* R = ct_fft_grouped<NZ, false, TZ, GS>(A, B, S, tw);
    C* O = (R == A) ? B : A;

    const Real hx = Real(g.hx), hy = Real(g.hy), hz = Real(g.hz);
    const Real fourpi = Real(4.0 * CUDART_PI);
    const bool tab = sp.tab_w != nullptr;
    const int my = signed_index(kyi, ny);
    Real flb = Real(0);      // 4 pi lambda_B = pois[s][s] / z_s^2 of a charged species
    for (int s = 0; s < S; ++s)
        if (sp.z[s] != Real(0)) { flb = sp.pois[s][s] / (sp.z[s] * sp.z[s]); break; }
    double e_acc = 0.0, q_acc = 0.0;
    for (int idx = threadIdx.x; idx < TILE; idx += kThreads) {
        const int kzi = idx / TZ, t = idx % TZ;
        const int pos = ct_gpos(kzi, TZ) + t;
        const int kxi = kx0 + t;
        const bool live = kxi < nxh;
        const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
        int m2 = 0;
        if (tab && live) { const int mz = signed_index(kzi, g.nz); m2 = kxi * kxi + my * my + mz * mz; }
        Real wr[DFT_TAB_W];
        Real kr[DFT_TAB_K], dkr[DFT_TAB_K];
        if (tab) {
            load_record(wr, sp.tab_w + (long long)m2 * sp.tab_ws, 2 * S);
            if (live) {
                load_record(kr, sp.tab_k + (long long)m2 * sp.tab_ks, Pn);
                if (GRAD) load_record(dkr, sp.tab_dk + (long long)m2 * sp.tab_ks, Pn);
            }
        }
        C v[DFT_MAXS];
#pragma unroll
        for (int s = 0; s < DFT_MAXS; ++s)
            if (s < S) v[s] = R[s * GS + pos];
        C acc[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) acc[a] = cmake<C>(Real(0), Real(0));
#pragma unroll
        for (int s = 0; s < DFT_MAXS; ++s) {
            if (s >= S) break;
            Real w0, j3;
            if (tab) { w0 = wr[2 * s]; j3 = wr[2 * s + 1]; }
            else fmt_weights<Real>(p.kmag, sp.R[s], &w0, &j3);
            const Real Rs = sp.R[s];
            acc[0] = cadd(acc[0], cscale(v[s], w0));
            acc[1] = cadd(acc[1], cscale(v[s], Rs * w0));
            acc[2] = cadd(acc[2], cscale(v[s], fourpi * Rs * Rs * w0));
            acc[3] = cadd(acc[3], cscale(v[s], fourpi * Rs * Rs * Rs * j3));
            acc[4] = cadd(acc[4], cscale(v[s], Rs * Rs * j3));       // w3 / (4 pi R)
        }
        if (live) {
            const Real inv_lap = inverse_laplacian<Real>(sp, g, p, kxi, kyi, kzi, hx, hy, hz);
            C dv[DFT_MAXS], es[DFT_MAXS];
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                if (s < S) {
                    dv[s] = v[s];
                    if (p.zero) dv[s].x -= sp.n_rho_b[s];       // DFT(rho - rho_bath) at k = 0
                }
                es[s] = cmake<C>(Real(0), Real(0));
            }
            const double wk = GRAD ? ((kxi == 0 || (g.nx % 2 == 0 && 2 * kxi == g.nx)) ? 1.0 : 2.0) : 0.0;
#pragma unroll
            for (int j = 0; j < DFT_MAXS; ++j) {
#pragma unroll
                for (int i = 0; i <= j; ++i) {
                    if (j >= S) continue;
                    Real K, dK = Real(0);
                    if (tab) {
                        K = kr[dft_pair(i, j)];
                        if (!p.zero) K -= sp.pois[i][j] * inv_lap;
                        if (GRAD) dK = dkr[dft_pair(i, j)];
                    } else {
                        K = es_kernel<Real>(sp, i, j, p, inv_lap, GRAD ? &dK : nullptr);
                    }
                    es[i] = cadd(es[i], cscale(dv[j], K));
                    if (j != i) es[j] = cadd(es[j], cscale(dv[i], K));
                    if constexpr (GRAD) {
                        const double re = double(dv[i].x) * dv[j].x + double(dv[i].y) * dv[j].y;
                        q_acc += wk * double(dK) * re * (j != i ? 2.0 : 1.0);
                    }
                }
            }
            const long long o = (long long)kzi * zstride + col0 + t;
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                if (s >= S) break;
                if constexpr (GRAD) e_acc += wk * (double(dv[s].x) * es[s].x + double(dv[s].y) * es[s].y);
                slot_es[(long long)s * g.nc + o] = es[s];
            }
            if (want_psi) {
                C q = cmake<C>(Real(0), Real(0));
#pragma unroll
                for (int s = 0; s < DFT_MAXS; ++s)
                    if (s < S) q = cadd(q, cscale(v[s], sp.z[s]));
                // psi_hat = 4 pi lambda_B q_hat / lap
                slot_es[(long long)S * g.nc + o] = cscale(q, flb * inv_lap);
            }
        }
        // the nine weighted-density spectra, 1/N applied (DFT_NSPEC order)
        store_wd_spectra<Real>(O, GS, pos, acc, sp.inv_n, p);
    }
    if constexpr (GRAD) {
        const double be = block_sum(e_acc, scratch_d);
        const double bq = block_sum(q_acc, scratch_d);
        if (threadIdx.x == 0) {
            const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            red_energy[2 * b] = be;
            red_energy[2 * b + 1] = bq;
        }
    }
    __syncthreads();
    C* Q = ct_fft_grouped<NZ, true, TZ, GS>(O, R, DFT_NSPEC, tw);
    tiles_store_grouped<TZ, NZ>(slot_n + col0, Q, g.nc, DFT_NSPEC, zstride, nxh - kx0);
}

// Second-half z pass (same contract as k_zconv_bwd): the ten Phi' spectra in (flags & 1), the
// bulk-fluid/Poisson spectra mixed in (flags & 2), ncomp_out one-body correlation spectra out.
// The points of a thread are handled together so that all of their global and table loads are
// in flight at once.
template <typename Real, int NZ, int TZ>
__global__ void __launch_bounds__(kThreads, 2) k_zconv_bwd_g(GridDesc g, SpeciesDesc<Real> sp, Real kfx, Real kfy,
                                                             Real kfz, int flags, int ncomp_out,
                                                             const Ctl* __restrict__ ctl,
                                                             typename Cplx<Real>::type* phi,
                                                             const typename Cplx<Real>::type* esA,
                                                             const typename Cplx<Real>::type* esB,
                                                             typename Cplx<Real>::type* es_mat,
                                                             const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    constexpr int TILE = TZ * NZ;
    constexpr int GS = ct_gstride(NZ, TZ, int(sizeof(C)));
    constexpr int PER = (TILE + kThreads - 1) / kThreads;
    constexpr int EMAX = DFT_MAXS + 1;
    extern __shared__ unsigned char smem_raw[];
    const int ny = g.ny, nxh = g.nxh, S = sp.S;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + NZ;
    C* B = A + DFT_NSPEC * GS;
    for (int i = threadIdx.x; i < NZ; i += kThreads) tw[i] = twz[i];
    const int kx0 = blockIdx.x * TZ;
    const int kyi = blockIdx.y;
    const long long zstride = (long long)ny * g.pxh;
    const long long col0 = (long long)kyi * g.pxh + kx0;
    const bool hs = (flags & 1) != 0, es_on = (flags & 2) != 0;
    const Real wA = CtlW<Real>::wA(ctl), wB = CtlW<Real>::wB(ctl);
    C* R = A;
    if (hs) {
        tiles_load_grouped<TZ, NZ, DFT_NSPEC>(A, phi + col0, g.nc, DFT_NSPEC, zstride, nxh - kx0);
        __syncthreads();
        R = ct_fft_grouped<NZ, false, TZ, GS>(A, B, DFT_NSPEC, tw);
    }
    C* O = (R == A) ? B : A;
    const Real fourpi = Real(4.0 * CUDART_PI);
    const bool tab = sp.tab_w != nullptr;
    const int my = signed_index(kyi, ny);

    // loads first: bulk-fluid/Poisson spectra and table records of all of this thread's points
    C ea[PER][EMAX];
    Real wr[PER][DFT_TAB_W];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        const int kzi = idx / TZ, t = idx % TZ;
        const int kxi = kx0 + t;
        const bool in_tile = (TILE % kThreads == 0) || idx < TILE;
        const bool live = in_tile && kxi < nxh;
        const long long o = (long long)kzi * zstride + col0 + t;
#pragma unroll
        for (int s = 0; s < EMAX; ++s) {
            ea[i][s] = cmake<C>(Real(0), Real(0));
            if (es_on && live && s < ncomp_out) {
                C e = cscale(esA[(long long)s * g.nc + o], wA);
                if (esB) e = cadd(e, cscale(esB[(long long)s * g.nc + o], wB));
                ea[i][s] = e;
            }
        }
        if (hs && tab) {
            int m2 = 0;
            if (live) { const int mz = signed_index(kzi, g.nz); m2 = kxi * kxi + my * my + mz * mz; }
            load_record(wr[i], sp.tab_w + (long long)m2 * sp.tab_ws, 2 * S);
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        if ((TILE % kThreads != 0) && idx >= TILE) break;
        const int kzi = idx / TZ, t = idx % TZ;
        const int pos = ct_gpos(kzi, TZ) + t;
        const int kxi = kx0 + t;
        C out[EMAX];
#pragma unroll
        for (int s = 0; s < EMAX; ++s) out[s] = ea[i][s];
        if (es_on && es_mat && kxi < nxh) {
            const long long o = (long long)kzi * zstride + col0 + t;
#pragma unroll
            for (int s = 0; s < EMAX; ++s)
                if (s < ncomp_out) es_mat[(long long)s * g.nc + o] = ea[i][s];
        }
        if (hs) {
            const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
            C asum[5];
            bwd_sums<Real>(R, GS, pos, p, asum);
            const C a0 = asum[0], a1 = asum[1], a2 = asum[2], a3 = asum[3], a4 = asum[4];
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                if (s >= S) break;
                Real w0, j3;
                const Real Rs = sp.R[s];
                if (tab) { w0 = wr[i][2 * s]; j3 = wr[i][2 * s + 1]; }
                else fmt_weights<Real>(p.kmag, Rs, &w0, &j3);
                C mu = cscale(a0, w0);
                mu = cadd(mu, cscale(a1, Rs * w0));
                mu = cadd(mu, cscale(a2, fourpi * Rs * Rs * w0));
                mu = cadd(mu, cscale(a3, fourpi * Rs * Rs * Rs * j3));
                mu = cadd(mu, cscale(a4, Rs * Rs * j3));
                out[s] = cmake<C>(out[s].x - mu.x, out[s].y - mu.y);
            }
        }
#pragma unroll
        for (int s = 0; s < EMAX; ++s)
            if (s < ncomp_out) O[s * GS + pos] = cscale(out[s], sp.inv_n);
    }
    __syncthreads();
    C* Q = ct_fft_grouped<NZ, true, TZ, GS>(O, R, ncomp_out, tw);
    tiles_store_grouped<TZ, NZ>(phi + col0, Q, g.nc, ncomp_out, zstride, nxh - kx0);
}

// ------------------------------------------------------------------------------------
// First-half z pass with TMA tiles (same contract as k_zconv_fwd without the grand-potential
// sums), persistent like k_zconv_bwd_tma: two stages of S species tiles are filled by TMA loads
// while the previous tile is transformed; seven weighted-density spectra are transformed back
// (zgroup order), the two y derivatives formed from m and n3 after that, and the nine leave
// through TMA stores, the bulk-fluid/Poisson spectra through plain stores.  A tensor map views a half-spectrum
// array as (x: nxh * E, y: ny, plane: nz * ncomp) 8-byte elements; a tile is the box
// (TZ * E, 1, NZ) at plane c * nz.  A wait that runs out sets DEV_TIMEOUT and the CTA stops
// after draining the loads it has in flight.
// Shared memory: stage 0 | stage 1 (S padded groups each) | W | V (nine padded groups each) |
// twiddles | two mbarriers.
// ------------------------------------------------------------------------------------
template <typename Real, int NZ, int TZ> __host__ __device__ constexpr size_t zfwd_tma_smem(int S) {
    using C = typename Cplx<Real>::type;
    constexpr size_t GS = size_t(ct_gstride(NZ, TZ, int(sizeof(C))));
    return ((2 * size_t(S) + 2 * DFT_NSPEC) * GS + NZ) * sizeof(C) + 2 * sizeof(uint64_t) + 128;
}

template <typename Real, int NZ, int TZ, int NT, int MINB, int SM = DFT_MAXS>
__global__ void __launch_bounds__(NT, MINB) k_zconv_fwd_tma(const __grid_constant__ CUtensorMap map_in,
                                                                         const __grid_constant__ CUtensorMap map_n,
                                                                         GridDesc g, SpeciesDesc<Real> sp, Real kfx,
                                                                         Real kfy, Real kfz, int want_psi,
                                                                         typename Cplx<Real>::type* __restrict__ slot_es,
                                                                         int ntiles_x, int ntiles,
                                                                         int* __restrict__ status,
                                                                         const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    constexpr int E = int(sizeof(C) / 8);
    constexpr int TILE = TZ * NZ;
    constexpr int GS = ct_gstride(NZ, TZ, int(sizeof(C)));
    constexpr int PER = (TILE + NT - 1) / NT;
    constexpr uint32_t BOX = uint32_t(TILE * sizeof(C));
    static_assert(NZ > 0 && NZ <= 256 && (TZ * sizeof(C)) % 16 == 0 && BOX % 128 == 0, "z TMA tile");
    extern __shared__ unsigned char smem_raw[];
    const int S = sp.S, ny = g.ny, nxh = g.nxh;
    const int Pn = S * (S + 1) / 2;
    const int stage_elems = S * GS;
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127);
    C* const stage0 = reinterpret_cast<C*>(base);
    C* W = stage0 + 2 * stage_elems;
    C* Vb = W + DFT_NSPEC * GS;
    C* tw = Vb + DFT_NSPEC * GS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + NZ);
    const uint32_t tile_bytes = uint32_t(S) * BOX;
    const long long zstride = (long long)ny * g.pxh;

    auto issue = [&](int tile, int s) {
        C* st = stage0 + s * stage_elems;
        const int x = (tile % ntiles_x) * TZ * E, y = tile / ntiles_x;
        tma::mbar_expect_tx(&bar[s], tile_bytes);
        for (int c = 0; c < S; ++c) tma::load_3d(st + c * GS, &map_in, x, y, c * NZ, &bar[s]);
    };
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < NZ; i += NT) tw[i] = twz[i];
    __syncthreads();
    int issued = 0, consumed = 0;   // per stage, packed (stage 1 << 16) | stage 0; thread 0
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            const int tile = blockIdx.x + s * gridDim.x;
            if (tile < ntiles) { issue(tile, s); issued += 1 << (16 * s); }
        }
    }
    const Real hx = Real(g.hx), hy = Real(g.hy), hz = Real(g.hz);
    const Real fourpi = Real(4.0 * CUDART_PI);
    const bool tab = sp.tab_w != nullptr;
    Real flb = Real(0);      // 4 pi lambda_B = pois[s][s] / z_s^2 of a charged species
    for (int s = 0; s < S; ++s)
        if (sp.z[s] != Real(0)) { flb = sp.pois[s][s] / (sp.z[s] * sp.z[s]); break; }
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int cur = it & 1;
        const int kx0 = (tile % ntiles_x) * TZ, kyi = tile / ntiles_x;
        const int my = signed_index(kyi, ny);
        // table records of this thread's points, in flight while the tile arrives
        // (the first point's; a thread's later points load theirs at the top of their iteration)
        Real wr[SM <= 3 ? 8 : DFT_TAB_W];
        Real kr[SM <= 3 ? 8 : DFT_TAB_K];
        auto load_tab = [&](int idx) {
            const int kxi = kx0 + idx % TZ;
            const int m2 = (((TILE % NT == 0) || idx < TILE) && kxi < nxh) ? kmode2(kxi, my, idx / TZ, g.nz) : 0;
            load_record(wr, sp.tab_w + (long long)m2 * sp.tab_ws, 2 * S);
            load_record(kr, sp.tab_k + (long long)m2 * sp.tab_ks, Pn);
        };
        if (tab) load_tab(threadIdx.x);
        const bool ok = tma::mbar_wait(&bar[cur], (it >> 1) & 1);
        // the previous tile's TMA stores have finished reading shared memory
        if (threadIdx.x == 0) tma::wait_read_all();
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, DEV_TIMEOUT);
                for (int s = 0; s < 2; ++s) {
                    const int n_is = (issued >> (16 * s)) & 0xffff, n_co = (consumed >> (16 * s)) & 0xffff;
                    if (n_is > n_co) tma::mbar_wait(&bar[s], (n_is - 1) & 1);
                }
            }
            break;
        }
        consumed += 1 << (16 * cur);
        C* st = stage0 + cur * stage_elems;
        C* X = ct_fft_grouped<NZ, false, TZ, GS, true, false, NT>(st, Vb, S, tw);
#pragma unroll 1
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if ((TILE % NT != 0) && idx >= TILE) break;
            if (tab && i > 0) load_tab(idx);
            const int kzi = idx / TZ, t = idx % TZ;
            const int pos = ct_gpos(kzi, TZ) + t;
            const int kxi = kx0 + t;
            const bool live = kxi < nxh;
            const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
            C v[SM];
#pragma unroll
            for (int s = 0; s < SM; ++s)
                if (s < S) v[s] = X[s * GS + pos];
            C acc[5];
#pragma unroll
            for (int a = 0; a < 5; ++a) acc[a] = cmake<C>(Real(0), Real(0));
#pragma unroll
            for (int s = 0; s < SM; ++s) {
                if (s >= S) break;
                Real w0, j3;
                if (tab) { w0 = wr[2 * s]; j3 = wr[2 * s + 1]; }
                else fmt_weights<Real>(p.kmag, sp.R[s], &w0, &j3);
                const Real Rs = sp.R[s];
                acc[0] = cadd(acc[0], cscale(v[s], w0));
                acc[1] = cadd(acc[1], cscale(v[s], Rs * w0));
                acc[2] = cadd(acc[2], cscale(v[s], fourpi * Rs * Rs * w0));
                acc[3] = cadd(acc[3], cscale(v[s], fourpi * Rs * Rs * Rs * j3));
                acc[4] = cadd(acc[4], cscale(v[s], Rs * Rs * j3));       // w3 / (4 pi R)
            }
            if (live) {
                const Real inv_lap = inverse_laplacian<Real>(sp, g, p, kxi, kyi, kzi, hx, hy, hz);
                C dv[SM], es[SM];
#pragma unroll
                for (int s = 0; s < SM; ++s) {
                    if (s < S) {
                        dv[s] = v[s];
                        if (p.zero) dv[s].x -= sp.n_rho_b[s];       // DFT(rho - rho_bath) at k = 0
                    }
                    es[s] = cmake<C>(Real(0), Real(0));
                }
#pragma unroll
                for (int j = 0; j < SM; ++j) {
#pragma unroll
                    for (int i2 = 0; i2 <= j; ++i2) {
                        if (j >= S) continue;
                        Real K;
                        if (tab) {
                            K = kr[dft_pair(i2, j)];
                            if (!p.zero) K -= sp.pois[i2][j] * inv_lap;
                        } else {
                            K = es_kernel<Real>(sp, i2, j, p, inv_lap, nullptr);
                        }
                        es[i2] = cadd(es[i2], cscale(dv[j], K));
                        if (j != i2) es[j] = cadd(es[j], cscale(dv[i2], K));
                    }
                }
                const long long o = (long long)kzi * zstride + (long long)kyi * g.pxh + kxi;
#pragma unroll
                for (int s = 0; s < SM; ++s)
                    if (s < S) slot_es[(long long)s * g.nc + o] = es[s];
                if (want_psi) {
                    C q = cmake<C>(Real(0), Real(0));
#pragma unroll
                    for (int s = 0; s < SM; ++s)
                        if (s < S) q = cadd(q, cscale(v[s], sp.z[s]));
                    slot_es[(long long)S * g.nc + o] = cscale(q, flb * inv_lap);
                }
            }
            // the weighted-density spectra but the y derivatives, 1/N applied
            store_wd_spectra_z<Real>(W, GS, pos, acc, sp.inv_n, p);
        }
        __syncthreads();
        // the stage is free now: refill it with the tile after next while the inverse runs
        if (threadIdx.x == 0) {
            const int next = tile + 2 * gridDim.x;
            if (next < ntiles) { issue(next, cur); issued += 1 << (16 * cur); }
        }
        C* Q = ct_fft_grouped<NZ, true, TZ, GS, false, true, NT>(W, Vb, kZGroups, tw);
        const bool nyq_y = (ny % 2 == 0) && (2 * kyi == ny);
        zfwd_add_y_derivatives<Real, TILE, NT>(Q, GS, nyq_y ? Real(0) : kval<Real>(kyi, ny, kfy));
        tma::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int a = 0; a < DFT_NSPEC; ++a) tma::store_3d(&map_n, kx0 * E, kyi, a * NZ, Q + zgroup(a) * GS);
            tma::commit();
        }
    }
    if (threadIdx.x == 0) tma::wait_all();
}

// ------------------------------------------------------------------------------------
// The k-space products of the first half as a pass of their own (the split first-half z stage:
// z forward transform of the S species, this pass, z inverse transform of the nine weighted
// densities).  At each k point of the S species spectra (after the x, y and z forward
// transforms) the nine weighted-density spectra, 1/N applied, into slot_n and the S
// bulk-fluid/Poisson spectra into slot_es, both in (kx, ky, kz); the same arithmetic per point as
// k_zconv_fwd_tma.  One thread per k point, kx fastest.
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kThreads, sizeof(Real) == 4 ? 3 : 2) k_zmul(GridDesc g, SpeciesDesc<Real> sp, Real kfx, Real kfy, Real kfz,
                                                   const typename Cplx<Real>::type* __restrict__ in,
                                                   typename Cplx<Real>::type* __restrict__ slot_n,
                                                   typename Cplx<Real>::type* __restrict__ slot_es) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    const int S = sp.S, nxh = g.nxh;
    const int Pn = S * (S + 1) / 2;
    const long long npt = (long long)g.nz * g.ny * nxh;
    const Real hx = Real(g.hx), hy = Real(g.hy), hz = Real(g.hz);
    const Real fourpi = Real(4.0 * CUDART_PI);
    const bool tab = sp.tab_w != nullptr;
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; q < npt; q += (long long)gridDim.x * kThreads) {
        const int kxi = int(q % nxh);
        const long long rz = q / nxh;
        const int kyi = int(rz % g.ny), kzi = int(rz / g.ny);
        const long long o = rz * g.pxh + kxi;
        const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
        const int m2 = tab ? kmode2(kxi, signed_index(kyi, g.ny), kzi, g.nz) : 0;
        C v[DFT_MAXS];
#pragma unroll
        for (int s = 0; s < DFT_MAXS; ++s)
            if (s < S) v[s] = in[(long long)s * g.nc + o];
        {   // the nine weighted-density spectra, 1/N applied (DFT_NSPEC order), as store_wd_spectra
            Real wr[DFT_TAB_W];
            if (tab) load_record(wr, sp.tab_w + (long long)m2 * sp.tab_ws, 2 * S);
            C acc[5];
#pragma unroll
            for (int a = 0; a < 5; ++a) acc[a] = cmake<C>(Real(0), Real(0));
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                if (s >= S) break;
                Real w0, j3;
                if (tab) { w0 = wr[2 * s]; j3 = wr[2 * s + 1]; }
                else fmt_weights<Real>(p.kmag, sp.R[s], &w0, &j3);
                const Real Rs = sp.R[s];
                acc[0] = cadd(acc[0], cscale(v[s], w0));
                acc[1] = cadd(acc[1], cscale(v[s], Rs * w0));
                acc[2] = cadd(acc[2], cscale(v[s], fourpi * Rs * Rs * w0));
                acc[3] = cadd(acc[3], cscale(v[s], fourpi * Rs * Rs * Rs * j3));
                acc[4] = cadd(acc[4], cscale(v[s], Rs * Rs * j3));       // w3 / (4 pi R)
            }
            store_wd_spectra<Real>(slot_n, int(g.nc), int(o), acc, sp.inv_n, p);
        }
        // the bulk-fluid/Poisson spectra
        Real kr[DFT_TAB_K];
        if (tab) load_record(kr, sp.tab_k + (long long)m2 * sp.tab_ks, Pn);
        const Real inv_lap = inverse_laplacian<Real>(sp, g, p, kxi, kyi, kzi, hx, hy, hz);
        C es[DFT_MAXS];
#pragma unroll
        for (int s = 0; s < DFT_MAXS; ++s) {
            if (s < S && p.zero) v[s].x -= sp.n_rho_b[s];       // DFT(rho - rho_bath) at k = 0
            es[s] = cmake<C>(Real(0), Real(0));
        }
#pragma unroll
        for (int j = 0; j < DFT_MAXS; ++j) {
#pragma unroll
            for (int i2 = 0; i2 <= j; ++i2) {
                if (j >= S) continue;
                Real K;
                if (tab) {
                    K = kr[dft_pair(i2, j)];
                    if (!p.zero) K -= sp.pois[i2][j] * inv_lap;
                } else {
                    K = es_kernel<Real>(sp, i2, j, p, inv_lap, nullptr);
                }
                es[i2] = cadd(es[i2], cscale(v[j], K));
                if (j != i2) es[j] = cadd(es[j], cscale(v[i2], K));
            }
        }
#pragma unroll
        for (int s = 0; s < DFT_MAXS; ++s)
            if (s < S) slot_es[(long long)s * g.nc + o] = es[s];
    }
}

// ------------------------------------------------------------------------------------
// Second-half z pass with TMA tiles (same contract as k_zconv_bwd), persistent: CTA b handles
// tiles b, b + gridDim.x, ...  Two shared-memory stages, each holding one tile's nine Phi'
// spectra (in zgroup order), are filled by TMA loads (one cp.async.bulk.tensor per component,
// completing on the stage's mbarrier) while the previous tile is transformed (seven groups: the
// y-derivative spectra folded into groups 3 and 4 by the first stage); the tile's bulk-fluid/Poisson
// spectra arrive in one single-buffered area (third mbarrier), loaded while the previous tile's
// inverse and this tile's forward transform run.  The ncomp_out results are written over the
// first groups of the transformed tile and leave through TMA stores.  At length 256 both
// transforms run in place (ct_fft_grouped_ip), which keeps the CTA within half an SM's shared
// memory (two CTAs per SM instead of one); shorter lengths, where two CTAs fit anyway,
// alternate with a scratch area W (one barrier per stage instead of two).  A tensor map views a
// half-spectrum array as (x: nxh * E, y: ny, plane: nz * ncomp) 8-byte elements, E =
// sizeof(complex) / 8; a component tile is the box (TZ * E, 1, NZ) at plane c * nz.  Columns
// past nxh read as zero and are not written.  The results go to map_out (map_phi's array for a
// single evaluation).  pair: the two line-search samples in one pass, each tile taken for both in
// turn: sample m's Phi' spectra are components 9 m .. 9 m + 8 of map_phi, its mixing weights
// ctl[m], its results components m ncomp_out .. of map_out, and the tile's ES spectra serve both.
// A tile's components are read and written only by the CTA that takes it, loads before stores,
// so map_out may overlap map_phi.  A wait that runs out sets DEV_TIMEOUT and the CTA stops after
// draining the loads it has in flight.
// Shared memory: stage 0 | stage 1 (nine padded groups each) | W (nine padded groups, below
// length 256) | ES (nes dense tiles) | twiddles | three mbarriers.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr bool zbwd_in_place(int nz) { return nz >= 256; }

template <typename Real, int NZ, int TZ> __host__ __device__ constexpr size_t zbwd_tma_smem(int nes) {
    using C = typename Cplx<Real>::type;
    constexpr size_t GS = size_t(ct_gstride(NZ, TZ, int(sizeof(C))));
    constexpr size_t groups = (zbwd_in_place(NZ) ? 2 : 3) * size_t(DFT_NSPEC);
    return (groups * GS + size_t(nes) * TZ * NZ + NZ) * sizeof(C) + 3 * sizeof(uint64_t) + 128;
}

template <typename Real, int NZ, int TZ, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_zconv_bwd_tma(const __grid_constant__ CUtensorMap map_phi,
                                                            const __grid_constant__ CUtensorMap map_esA,
                                                            const __grid_constant__ CUtensorMap map_esB,
                                                            const __grid_constant__ CUtensorMap map_out, GridDesc g,
                                                            SpeciesDesc<Real> sp, Real kfx, Real kfy, Real kfz,
                                                            int flags, int ncomp_out, int has_esB, int pair,
                                                            const Ctl* __restrict__ ctl,
                                                            typename Cplx<Real>::type* es_mat, int ntiles_x,
                                                            int ntiles, int* __restrict__ status,
                                                            const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    constexpr int E = int(sizeof(C) / 8);
    constexpr int TILE = TZ * NZ;
    constexpr int GS = ct_gstride(NZ, TZ, int(sizeof(C)));
    constexpr int PER = (TILE + NT - 1) / NT;
    constexpr int EMAX = DFT_MAXS + 1;
    constexpr uint32_t BOX = uint32_t(TILE * sizeof(C));
    static_assert(NZ > 0 && NZ <= 256 && (TZ * sizeof(C)) % 16 == 0 && BOX % 128 == 0, "z TMA tile");
    extern __shared__ unsigned char smem_raw[];
    const bool hs = (flags & 1) != 0, es_on = (flags & 2) != 0;
    const int nes = es_on ? ncomp_out * (has_esB ? 2 : 1) : 0;
    constexpr int stage_elems = DFT_NSPEC * GS;
    constexpr bool IP = zbwd_in_place(NZ);
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127);
    C* const stage0 = reinterpret_cast<C*>(base);
    C* const W = stage0 + 2 * stage_elems;
    C* const es_t = W + (IP ? 0 : stage_elems);
    C* tw = es_t + nes * TILE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + NZ);
    const int S = sp.S, ny = g.ny, nxh = g.nxh;
    const long long zstride = (long long)ny * g.pxh;
    // Work items: tiles, or (pair) each tile twice, for the two line-search samples in turn
    // (sample m's nine Phi' spectra at components 9 m .. 9 m + 8 of map_phi, its weights in
    // ctl[m], its results to components m ncomp_out .. of map_out); the ES tiles of a tile are
    // loaded once for both.
    const int shift = pair ? 1 : 0;
    auto item_tile = [&](int item) { return blockIdx.x + (item >> shift) * gridDim.x; };

    auto issue_phi = [&](int item, int s) {
        C* st = stage0 + s * stage_elems;
        const int tile = item_tile(item), m = pair ? (item & 1) : 0;
        const int x = (tile % ntiles_x) * TZ * E, y = tile / ntiles_x;
        tma::mbar_expect_tx(&bar[s], uint32_t(DFT_NSPEC) * BOX);
        for (int c = 0; c < DFT_NSPEC; ++c)
            tma::load_3d(st + zgroup(c) * GS, &map_phi, x, y, (m * DFT_NSPEC + c) * NZ, &bar[s]);
    };
    auto issue_es = [&](int tile) {
        const int x = (tile % ntiles_x) * TZ * E, y = tile / ntiles_x;
        tma::mbar_expect_tx(&bar[2], uint32_t(nes) * BOX);
        for (int c = 0; c < ncomp_out; ++c) tma::load_3d(es_t + c * TILE, &map_esA, x, y, c * NZ, &bar[2]);
        if (has_esB)
            for (int c = 0; c < ncomp_out; ++c)
                tma::load_3d(es_t + (ncomp_out + c) * TILE, &map_esB, x, y, c * NZ, &bar[2]);
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) tma::mbar_init(&bar[b], 1);
        tma::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < NZ; i += NT) tw[i] = twz[i];
    __syncthreads();
    // Phi' loads issued / consumed per stage, packed as (stage 1 << 16) | stage 0, and ES loads
    // issued / consumed; meaningful in thread 0
    int issued = 0, consumed = 0, es_issued = 0, es_consumed = 0;
    if (threadIdx.x == 0) {
        if (hs)
            for (int s = 0; s < 2; ++s)
                if (item_tile(s) < ntiles) { issue_phi(s, s); issued += 1 << (16 * s); }
        if (es_on && blockIdx.x < ntiles) { issue_es(blockIdx.x); ++es_issued; }
    }
    // on a wait that ran out: record it, let the copies in flight land, stop
    auto drain = [&]() {
        if (threadIdx.x == 0) {
            atomicOr(status, DEV_TIMEOUT);
            for (int s = 0; s < 2; ++s) {
                const int n_is = (issued >> (16 * s)) & 0xffff, n_co = (consumed >> (16 * s)) & 0xffff;
                if (n_is > n_co) tma::mbar_wait(&bar[s], (n_is - 1) & 1);
            }
            if (es_issued > es_consumed) tma::mbar_wait(&bar[2], (es_issued - 1) & 1);
        }
    };
    const Real fourpi = Real(4.0 * CUDART_PI);
    const bool tab = sp.tab_w != nullptr;
    for (int it = 0;; ++it) {
        const int tile = item_tile(it);
        if (tile >= ntiles) break;
        const int m = pair ? (it & 1) : 0;
        const int ti = it >> shift;                 // this CTA's tile count so far
        const bool last_of_tile = !pair || m == 1;
        const Real wA = CtlW<Real>::wA(ctl + m), wB = CtlW<Real>::wB(ctl + m);
        const int cur = it & 1;
        const int kx0 = (tile % ntiles_x) * TZ, kyi = tile / ntiles_x;
        const int my = signed_index(kyi, ny);
        // the first point's table record is in flight while the tile arrives; a thread's later
        // points load theirs where they are used
        Real wr[DFT_TAB_W];
        if (hs && tab) {
            const int idx = threadIdx.x;
            const int kxi = kx0 + idx % TZ;
            const int m2 = (((TILE % NT == 0) || idx < TILE) && kxi < nxh) ? kmode2(kxi, my, idx / TZ, g.nz) : 0;
            load_record(wr, sp.tab_w + (long long)m2 * sp.tab_ws, 2 * S);
        }
        C* const st = stage0 + cur * stage_elems;
        C* X = st;
        if (hs) {
            const bool ok = tma::mbar_wait(&bar[cur], (it >> 1) & 1);
            if (__syncthreads_or(!ok)) { drain(); break; }
            if (threadIdx.x == 0) consumed += 1 << (16 * cur);
            // the y derivatives folded into groups 3 and 4 on the way into the first stage: seven
            // groups transformed
            const bool nyq_y = (ny % 2 == 0) && (2 * kyi == ny);
            const C kf = cmake<C>(nyq_y ? Real(0) : kval<Real>(kyi, ny, kfy), Real(0));
            if constexpr (IP) ct_fft_grouped_ip<NZ, false, TZ, GS, true, false, NT, true>(X, kZGroups, tw, kf);
            else X = ct_fft_grouped<NZ, false, TZ, GS, true, false, NT, true>(st, W, kZGroups, tw, kf);
        }
        // the ES tiles of this tile (loaded since the previous tile's pointwise phase; a pair's
        // second item reuses them); the barrier also ends the forward transform
        const bool ok_es = (es_on && m == 0) ? tma::mbar_wait(&bar[2], ti & 1) : true;
        if (__syncthreads_or(!ok_es)) { drain(); break; }
        if (threadIdx.x == 0 && es_on && m == 0) ++es_consumed;
#pragma unroll 1
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if ((TILE % NT != 0) && idx >= TILE) break;
            const int kzi = idx / TZ, t = idx % TZ;
            const int pos = ct_gpos(kzi, TZ) + t;
            const int kxi = kx0 + t;
            C out[EMAX];
#pragma unroll
            for (int s = 0; s < EMAX; ++s) {
                out[s] = cmake<C>(Real(0), Real(0));
                if (es_on && s < ncomp_out) {
                    C e = cscale(es_t[s * TILE + idx], wA);
                    if (has_esB) e = cadd(e, cscale(es_t[(ncomp_out + s) * TILE + idx], wB));
                    out[s] = e;
                }
            }
            if (es_on && es_mat && kxi < nxh) {
                const long long o = (long long)kzi * zstride + (long long)kyi * g.pxh + kxi;
#pragma unroll
                for (int s = 0; s < EMAX; ++s)
                    if (s < ncomp_out) es_mat[(long long)s * g.nc + o] = out[s];
            }
            if (hs) {
                if (i > 0 && tab)
                    load_record(wr, sp.tab_w + (long long)(kxi < nxh ? kmode2(kxi, my, kzi, g.nz) : 0) * sp.tab_ws,
                                2 * S);
                const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
                C asum[5];
                bwd_sums_folded<Real>(X, GS, pos, p, asum);
                const C a0 = asum[0], a1 = asum[1], a2 = asum[2], a3 = asum[3], a4 = asum[4];
#pragma unroll
                for (int s = 0; s < DFT_MAXS; ++s) {
                    if (s >= S) break;
                    Real w0, j3;
                    const Real Rs = sp.R[s];
                    if (tab) { w0 = wr[2 * s]; j3 = wr[2 * s + 1]; }
                    else fmt_weights<Real>(p.kmag, Rs, &w0, &j3);
                    C mu = cscale(a0, w0);
                    mu = cadd(mu, cscale(a1, Rs * w0));
                    mu = cadd(mu, cscale(a2, fourpi * Rs * Rs * w0));
                    mu = cadd(mu, cscale(a3, fourpi * Rs * Rs * Rs * j3));
                    mu = cadd(mu, cscale(a4, Rs * Rs * j3));
                    out[s] = cmake<C>(out[s].x - mu.x, out[s].y - mu.y);
                }
            }
            // over the first groups at this thread's own position (read above, by this thread only)
#pragma unroll
            for (int s = 0; s < EMAX; ++s)
                if (s < ncomp_out) X[s * GS + pos] = cscale(out[s], sp.inv_n);
        }
        __syncthreads();
        // the ES area is free after a tile's last item: load the next tile's while this one is
        // finished
        if (threadIdx.x == 0 && es_on && last_of_tile) {
            const int next = tile + gridDim.x;
            if (next < ntiles) { issue_es(next); ++es_issued; }
        }
        C* Q = X;
        if constexpr (IP) ct_fft_grouped_ip<NZ, true, TZ, GS, false, true, NT>(X, ncomp_out, tw);
        else Q = ct_fft_grouped<NZ, true, TZ, GS, false, true, NT>(X, X == st ? W : st, ncomp_out, tw);
        tma::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int s = 0; s < ncomp_out; ++s)
                tma::store_3d(&map_out, kx0 * E, kyi, (m * ncomp_out + s) * NZ, Q + s * GS);
            tma::commit();
            // the stores read the stage or W: let them finish reading before either is written
            tma::wait_read_all();
            if (hs && item_tile(it + 2) < ntiles) { issue_phi(it + 2, cur); issued += 1 << (16 * cur); }
        }
    }
    if (threadIdx.x == 0) tma::wait_all();
}

// ------------------------------------------------------------------------------------
// Pointwise derivatives of eq. Phi; xi = |nV2|^2/n2^2 is clamped to [0, 1] (Sec. "Numerical
// Stability") and the xi terms vanish where n2 <= 1e-30.  log(1 - n3) and 1/(1 - n3)^m are
// formed in FP64 where n3 >= 0.5, i.e. where n3 approaches 1; below, 1 - n3 is exact in the
// working precision and log1p / the reciprocal are within 2 ulp.  Returns false if n3 >= 1.
// ------------------------------------------------------------------------------------
// White Bear g(n3) = (n3 + D^2 ln D) / n3^2 and g'(n3), D = 1 - n3 (the other forms' last term
// is (n2^3 - 3 n2 nV2.nV2) f(n3), f = g / (36 pi D^2) for White Bear).  Below n3 = 1/2 the closed
// form cancels, so the power series of ln D is summed: g = 3/2 - sum_{k>=3} 2 n3^(k-2) /
// (k (k-1) (k-2)), g' = -sum_{k>=3} 2 n3^(k-3) / (k (k-1)), to k = 24 (FP32) / 52 (FP64), where
// the truncation is below the working precision; from 1/2 up the closed form in FP64 with
// lnD_hi = ln D.
template <typename Real>
__device__ __forceinline__ void wb_g(Real n3, double lnD_hi, Real* g, Real* dg) {
    if (n3 < Real(0.5)) {
        constexpr int K = sizeof(Real) == 4 ? 24 : 52;
        Real sg = Real(0), sd = Real(0);
#pragma unroll
        for (int k = K; k >= 3; --k) {
            sg = sg * n3 + Real(2.0 / (double(k) * double(k - 1) * double(k - 2)));
            sd = sd * n3 + Real(2.0 / (double(k) * double(k - 1)));
        }
        *g = Real(1.5) - n3 * sg;
        *dg = -sd;
    } else {
        const double u = double(n3), d = 1.0 - u, num = u + d * d * lnD_hi;
        *g = Real(num / (u * u));
        *dg = Real((u - 2.0 * d * lnD_hi) / (u * u) - 2.0 * num / (u * u * u));
    }
}

// Phi itself (eq. Phi, or the form `kind`), in FP64, for the grand potential; same clamp as the
// derivatives.
template <typename Real> __device__ __forceinline__ double phi_value(const Real* n, int kind) {
    const double n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
    const double D = 1.0 - n3;
    const double q = double(n[7]) * n[7] + double(n[8]) * n[8] + double(n[9]) * n[9];
    const double dot = double(n[4]) * n[7] + double(n[5]) * n[8] + double(n[6]) * n[9];
    const double base = -n0 * log(D) + (n1 * n2 - dot) / D;
    if (kind == DFT_PHI_ROSENFELD) return base + (n2 * n2 * n2 - 3.0 * n2 * q) / (24.0 * CUDART_PI * D * D);
    if (kind == DFT_PHI_WHITE_BEAR) {
        double g, dg;
        wb_g<double>(n3, log(D), &g, &dg);
        return base + (n2 * n2 * n2 - 3.0 * n2 * q) * g / (36.0 * CUDART_PI * D * D);
    }
    double xi = (n2 > 1e-30) ? q / (n2 * n2) : 1.0;
    xi = xi < 0.0 ? 0.0 : (xi > 1.0 ? 1.0 : xi);
    const double om = 1.0 - xi;
    return base + n2 * n2 * n2 * om * om * om / (24.0 * CUDART_PI * D * D);
}

// The derivatives of eq. Phi (kind DFT_PHI_RSLT) or of the other forms, whose last term
// T f(n3), T = n2^3 - 3 n2 nV2.nV2, gives dPhi/dn2 += 3 (n2^2 - nV2.nV2) f, dPhi/dn3 += T f',
// dPhi/dnV2 += -6 n2 f nV2 (no clamp); f = 1/(24 pi D^2) (Rosenfeld) or g/(36 pi D^2) (White
// Bear, f' = (g' D + 2 g)/(36 pi D^3)).
template <typename Real> __device__ __forceinline__ bool phi_derivatives(Real* n, int kind) {
    const Real n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
    const Real v1x = n[4], v1y = n[5], v1z = n[6], v2x = n[7], v2y = n[8], v2z = n[9];
    Real lnD, fiD;
    double lnD_hi = 0.0;
    bool ok = true;
    if (n3 < Real(0.5)) {
        lnD = log1p(-n3);
        fiD = Real(1) / (Real(1) - n3);
    } else {
        const double D = 1.0 - double(n3);
        ok = D > 0.0;
        lnD_hi = log(D);
        lnD = Real(lnD_hi);
        fiD = Real(1.0 / D);
    }
    const Real fiD2 = fiD * fiD, fiD3 = fiD2 * fiD;
    const Real q = v2x * v2x + v2y * v2y + v2z * v2z;
    const Real dot = v1x * v2x + v1y * v2y + v1z * v2z;
    // the constant denominators as products with their reciprocals (rounded once, from double)
    const Real i4pi = Real(1.0 / (4.0 * CUDART_PI)), i8pi = Real(1.0 / (8.0 * CUDART_PI));
    const Real i12pi = Real(1.0 / (12.0 * CUDART_PI)), i24pi = Real(1.0 / (24.0 * CUDART_PI));
    const Real i36pi = Real(1.0 / (36.0 * CUDART_PI));
    n[0] = -lnD;
    n[1] = n2 * fiD;
    n[4] = -v2x * fiD;
    n[5] = -v2y * fiD;
    n[6] = -v2z * fiD;
    if (kind != DFT_PHI_RSLT) {
        Real f, df;
        if (kind == DFT_PHI_ROSENFELD) {
            f = fiD2 * i24pi;
            df = fiD3 * i12pi;
        } else {
            Real g, dg;
            wb_g<Real>(n3, lnD_hi, &g, &dg);
            f = g * fiD2 * i36pi;
            df = (dg * fiD2 + Real(2) * g * fiD3) * i36pi;
        }
        const Real T = n2 * n2 * n2 - Real(3) * n2 * q;
        const Real c6 = Real(6) * n2 * f;
        n[2] = n1 * fiD + Real(3) * (n2 * n2 - q) * f;
        n[3] = n0 * fiD + (n1 * n2 - dot) * fiD2 + T * df;
        n[7] = -v1x * fiD - c6 * v2x;
        n[8] = -v1y * fiD - c6 * v2y;
        n[9] = -v1z * fiD - c6 * v2z;
        return ok;
    }
    Real xi = (n2 > Real(1e-30)) ? q / (n2 * n2) : Real(1);
    xi = xi < Real(0) ? Real(0) : (xi > Real(1) ? Real(1) : xi);
    const Real om = Real(1) - xi;
    n[2] = n1 * fiD + n2 * n2 * om * om * (Real(1) + xi) * fiD2 * i8pi;
    n[3] = n0 * fiD + (n1 * n2 - dot) * fiD2 + n2 * n2 * n2 * om * om * om * fiD3 * i12pi;
    const Real cv = n2 * om * om * fiD2 * i4pi;
    n[7] = -v1x * fiD - cv * v2x;
    n[8] = -v1y * fiD - cv * v2y;
    n[9] = -v1z * fiD - cv * v2z;
    return ok;
}

// The ten weighted densities in the x passes: five complex lines of two real rows each,
// (n0, n1), (n2, nV1y), (n3, nV2x), (nV1x, nV1z), (nV2y, nV2z) (line 2 carries n3 and
// nV2x = i k_x n3, line 3 nV1x = i k_x m; on the way back, line 2 gives B3 and line 3 B4).
// wd_comp(l, j): component of slot j of line l; wd_line / wd_slot: the inverse.
__host__ __device__ constexpr int wd_comp(int l, int j) {
    return l == 0 ? j : (l == 1 ? (j ? 5 : 2) : (l == 2 ? (j ? 7 : 3) : (l == 3 ? (j ? 6 : 4) : 8 + j)));
}
__host__ __device__ constexpr int wd_line(int c) {
    return c < 2 ? 0 : (c == 2 || c == 5 ? 1 : (c == 3 || c == 7 ? 2 : (c == 4 || c == 6 ? 3 : 4)));
}
__host__ __device__ constexpr int wd_slot(int c) { return (c == 1 || c == 5 || c == 7 || c == 6 || c == 9) ? 1 : 0; }

// Load the Hermitian half rows of two components (mixed wA * A + wB * B) as Z = a + i b over the
// full length nx (Z[nx-k] = conj(a_k) + i conj(b_k)).  Optionally stores the mixed half rows.
// Items in flight per thread in the update pass's pointwise phase (build flag).
#ifndef DFT_XUPD_BATCH
#define DFT_XUPD_BATCH 1
#endif

// 16 bytes of consecutive real values (four floats or two doubles), for 16-byte loads and stores.
template <typename Real> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ float4 ld16(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ double2 ld16(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st16(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st16(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
__device__ __forceinline__ float& vel(float4& v, int e) { return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w)); }
__device__ __forceinline__ double& vel(double2& v, int e) { return e == 0 ? v.x : v.y; }
template <typename V> __device__ __forceinline__ V vzero() { V v; memset(&v, 0, sizeof(V)); return v; }

// Loads are issued in batches of kBatch elements per thread before any store, so that several
// are in flight at once.
template <typename Real, int NX>
__device__ __forceinline__ void load_pair_rows(const GridDesc& g, int lines, int lines_per_row, long long row0,
                                               long long nrows, int ncomp,
                                               const typename Cplx<Real>::type* A,
                                               const typename Cplx<Real>::type* Bm, Real wA, Real wB,
                                               typename Cplx<Real>::type* mat_out,
                                               typename Cplx<Real>::type* dst) {
    using C = typename Cplx<Real>::type;
    constexpr int kBatch = 4;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const bool even = (nx % 2) == 0;
    const int total = lines * nxh;
    for (int base = threadIdx.x; base < total; base += kBatch * kThreads) {
        C av[kBatch], bv[kBatch], aB[kBatch], bB[kBatch];
        long long oa[kBatch], ob[kBatch];
        bool live[kBatch], hasb[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
            const long long row = row0 + l / lines_per_row;
            const int ca = 2 * (l % lines_per_row), cb = ca + 1;
            live[j] = idx < total && row < nrows;
            hasb[j] = cb < ncomp;
            oa[j] = (long long)ca * g.nc + row * g.pxh + k;
            ob[j] = (long long)cb * g.nc + row * g.pxh + k;
            av[j] = bv[j] = aB[j] = bB[j] = cmake<C>(Real(0), Real(0));
            if (live[j]) {
                av[j] = A[oa[j]];
                if (hasb[j]) bv[j] = A[ob[j]];
                if (Bm) {
                    aB[j] = Bm[oa[j]];
                    if (hasb[j]) bB[j] = Bm[ob[j]];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            if (idx >= total) continue;
            const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
            C a = cadd(cscale(av[j], wA), cscale(aB[j], wB));
            C b = cadd(cscale(bv[j], wA), cscale(bB[j], wB));
            if (k == 0 || (even && 2 * k == nx)) { a.y = Real(0); b.y = Real(0); }
            if (mat_out && live[j]) {
                mat_out[oa[j]] = a;
                if (hasb[j]) mat_out[ob[j]] = b;
            }
            dst[l * pitch + xo<NX>(k)] = cmake<C>(a.x - b.y, a.y + b.x);
            if (k != 0 && !(even && 2 * k == nx)) dst[l * pitch + xo<NX>(nx - k)] = cmake<C>(a.x + b.y, b.x - a.y);
        }
    }
}

// The S species' half rows of `rows` grid rows as ceil(S/2) complex lines each (species 2l and
// 2l + 1 in line l of a row's lines), for NM sets of spectra (spec, then spec2 into the lines
// after the first set's).  Items are (set, line, k), k fastest; each thread issues the loads of
// kBatch items before any store, so that they are in flight together.
template <typename Real, int NX, int NM = 1>
__device__ __forceinline__ void load_species_rows(const GridDesc& g, int rows, long long row0, long long nrows, int S,
                                                  const typename Cplx<Real>::type* __restrict__ spec,
                                                  const typename Cplx<Real>::type* __restrict__ spec2,
                                                  typename Cplx<Real>::type* dst) {
    using C = typename Cplx<Real>::type;
    constexpr int kBatch = 4;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const bool even = (nx % 2) == 0;
    const int lpr = (S + 1) / 2;
    const int lines = rows * lpr;                 // lines of one set
    const int total = NM * lines * nxh;
    for (int base = threadIdx.x; base < total; base += kBatch * kThreads) {
        C av[kBatch], bv[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            const int ml = idx / nxh, k = idx - (idx / nxh) * nxh;
            const int m = NM == 1 ? 0 : ml / lines, l = ml - m * lines;
            const long long row = row0 + l / lpr;
            const int ca = 2 * (l % lpr), cb = ca + 1;
            const C* src = (NM == 2 && m == 1) ? spec2 : spec;
            const long long o = row * g.pxh + k;
            av[j] = bv[j] = cmake<C>(Real(0), Real(0));
            if (idx < total && row < nrows) {
                av[j] = src[(long long)ca * g.nc + o];
                if (cb < S) bv[j] = src[(long long)cb * g.nc + o];
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            if (idx >= total) continue;
            const int ml = idx / nxh, k = idx - (idx / nxh) * nxh;
            C a = av[j], b = bv[j];
            const bool edge = k == 0 || (even && 2 * k == nx);
            if (edge) { a.y = Real(0); b.y = Real(0); }
            dst[ml * pitch + xo<NX>(k)] = cmake<C>(a.x - b.y, a.y + b.x);
            if (!edge) dst[ml * pitch + xo<NX>(nx - k)] = cmake<C>(a.x + b.y, b.x - a.y);
        }
    }
}

// One component's half rows of `rows` grid rows, two grid rows per complex line (rows 2l and
// 2l + 1 of the block in line l; a missing partner row reads as zero).
template <typename Real, int NX>
__device__ __forceinline__ void load_row_pairs(const GridDesc& g, int rows, long long row0, long long nrows,
                                               const typename Cplx<Real>::type* __restrict__ spec,
                                               typename Cplx<Real>::type* dst) {
    using C = typename Cplx<Real>::type;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const bool even = (nx % 2) == 0;
    const int lines = (rows + 1) / 2;
    const int total = lines * nxh;
    // the loads of kBatch items per thread in flight together
    constexpr int kBatch = 4;
    for (int base = threadIdx.x; base < total; base += kBatch * kThreads) {
        C av[kBatch], bv[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
            const int ra = 2 * l, rb = 2 * l + 1;
            av[j] = bv[j] = cmake<C>(Real(0), Real(0));
            if (idx < total) {
                if (row0 + ra < nrows) av[j] = spec[(row0 + ra) * g.pxh + k];
                if (rb < rows && row0 + rb < nrows) bv[j] = spec[(row0 + rb) * g.pxh + k];
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const int idx = base + j * kThreads;
            if (idx >= total) continue;
            const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
            C a = av[j], b = bv[j];
            const bool edge = k == 0 || (even && 2 * k == nx);
            if (edge) { a.y = Real(0); b.y = Real(0); }
            dst[l * pitch + xo<NX>(k)] = cmake<C>(a.x - b.y, a.y + b.x);
            if (!edge) dst[l * pitch + xo<NX>(nx - k)] = cmake<C>(a.x + b.y, b.x - a.y);
        }
    }
}

// The ten weighted-density rows of `rows` grid rows as five complex lines each (wd_comp
// arrangement), built from the nine kept spectra mixed as wA * A + wB * B (B optional), with
// n_V1x = i k_x m and n_V2x = i k_x n3 (zero on the Nyquist index); mat_out (optional) receives
// the nine mixed spectra.  One thread handles all lines of one (row, k): the index arithmetic is
// shared and its eighteen loads are in flight together.  NM mixtures (weights wA[a], wB[a]) of
// the same loads: mixture a of row r goes to lines (r NM + a) 5 .. + 4.
// STAGED: the spectra come from shared memory instead, component c of the block's rows at
// stage[c cstride + r pxh + k] (slot B's at components 9..17; Bm only tells that they are there).
template <typename Real, int NX, int NM = 1, bool STAGED = false>
__device__ __forceinline__ void load_wd_rows(const GridDesc& g, int rows, long long row0, long long nrows,
                                             const typename Cplx<Real>::type* A,
                                             const typename Cplx<Real>::type* Bm, const Real* wA,
                                             const Real* wB, typename Cplx<Real>::type* mat_out, Real kfx,
                                             typename Cplx<Real>::type* dst,
                                             const typename Cplx<Real>::type* stage = nullptr, int cstride = 0) {
    using C = typename Cplx<Real>::type;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const bool even = (nx % 2) == 0;
    for (int idx = threadIdx.x; idx < rows * nxh; idx += blockDim.x) {
        const int r = idx / nxh, k = idx - (idx / nxh) * nxh;
        const long long row = row0 + r;
        const bool live = row < nrows;
        const long long o = row * g.pxh + k;
        C v[DFT_NSPEC], vb[DFT_NSPEC];
#pragma unroll
        for (int c = 0; c < DFT_NSPEC; ++c) {
            v[c] = vb[c] = cmake<C>(Real(0), Real(0));
            if (live) {
                if constexpr (STAGED) {
                    v[c] = stage[c * cstride + r * g.pxh + k];
                    if (Bm) vb[c] = stage[(DFT_NSPEC + c) * cstride + r * g.pxh + k];
                } else {
                    v[c] = A[(long long)c * g.nc + o];
                    if (Bm) vb[c] = Bm[(long long)c * g.nc + o];
                }
            }
        }
        const bool edge = k == 0 || (even && 2 * k == nx);
        const bool nyq = even && 2 * k == nx;
        const Real kx = Real(k) * kfx;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            C u[DFT_NSPEC];
#pragma unroll
            for (int c = 0; c < DFT_NSPEC; ++c) {
                u[c] = cadd(cscale(v[c], wA[m]), cscale(vb[c], wB[m]));
                if (edge) u[c].y = Real(0);
                if (NM == 1 && mat_out && live) mat_out[(long long)c * g.nc + o] = u[c];
            }
            const C zero = cmake<C>(Real(0), Real(0));
            const C dm = nyq ? zero : cmake<C>(-kx * u[4].y, kx * u[4].x);     // i k_x m
            const C dn3 = nyq ? zero : cmake<C>(-kx * u[3].y, kx * u[3].x);    // i k_x n3
            // line l holds (a, b) = (wd_comp(l, 0), wd_comp(l, 1))
            const C la[5] = {u[0], u[2], u[3], dm, u[7]};
            const C lb[5] = {u[1], u[5], dn3, u[6], u[8]};
            const int l0 = (r * NM + m) * 5;
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                const C a = la[l], b = lb[l];
                dst[(l0 + l) * pitch + xo<NX>(k)] = cmake<C>(a.x - b.y, a.y + b.x);
                if (!edge) dst[(l0 + l) * pitch + xo<NX>(nx - k)] = cmake<C>(a.x + b.y, b.x - a.y);
            }
        }
    }
}

// Separate Z = FFT(a + i b) of two real rows into their half spectra and store them.
template <typename Real, int NX>
__device__ __forceinline__ void store_pair_rows(const GridDesc& g, int lines, int lines_per_row, long long row0,
                                                long long nrows, int ncomp, const typename Cplx<Real>::type* R,
                                                typename Cplx<Real>::type* out) {
    using C = typename Cplx<Real>::type;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    for (int idx = threadIdx.x; idx < lines * nxh; idx += blockDim.x) {
        const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
        const long long row = row0 + l / lines_per_row;
        if (row >= nrows) continue;
        const int ca = 2 * (l % lines_per_row), cb = ca + 1;
        const C zk = R[l * pitch + xo<NX>(k)];
        const C znk = R[l * pitch + xo<NX>(k == 0 ? 0 : nx - k)];
        const C s = cadd(zk, cconj(znk));
        const C d = csub(zk, cconj(znk));
        out[(long long)ca * g.nc + row * g.pxh + k] = cmake<C>(Real(0.5) * s.x, Real(0.5) * s.y);
        if (cb < ncomp) out[(long long)cb * g.nc + row * g.pxh + k] = cmake<C>(Real(0.5) * d.y, Real(-0.5) * d.x);
    }
}

// Half spectra of the ten dPhi/dn_alpha rows of `rows` grid rows (five complex lines each, in the
// wd_comp arrangement of load_pair_rows) into the nine spectra the y and z passes carry:
// Phi_0..Phi_2, B3 = Phi_3 - i k_x Phi_V2x, B4 = -i k_x Phi_V1x, Phi_V1y, Phi_V1z, Phi_V2y,
// Phi_V2z (the -i k_x terms dropped on the Nyquist index).  Each line maps to its own outputs:
// line 2 holds Phi_3 and Phi_V2x, line 3 Phi_V1x and Phi_V1z.
// NM mixtures: those of sub-row r NM + m (lines (r NM + m) 5 ..) go to out + m DFT_NSPEC nc.
template <typename Real, int NX, int NM = 1>
__device__ __forceinline__ void store_phi_spectra(const GridDesc& g, int rows, long long row0, long long nrows,
                                                  Real kfx, const typename Cplx<Real>::type* R,
                                                  typename Cplx<Real>::type* out0) {
    using C = typename Cplx<Real>::type;
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const bool even = (nx % 2) == 0;
    for (int idx = threadIdx.x; idx < rows * NM * nxh; idx += blockDim.x) {
        const int rr = idx / nxh, k = idx - (idx / nxh) * nxh;
        const int r = rr / NM;
        const long long row = row0 + r;
        if (row >= nrows) continue;
        C* out = out0 + (long long)(rr - r * NM) * DFT_NSPEC * g.nc;
        C a[5], b[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const C zk = R[(rr * 5 + l) * pitch + xo<NX>(k)];
            const C znk = R[(rr * 5 + l) * pitch + xo<NX>(k == 0 ? 0 : nx - k)];
            const C s = cadd(zk, cconj(znk));
            const C d = csub(zk, cconj(znk));
            a[l] = cmake<C>(Real(0.5) * s.x, Real(0.5) * s.y);
            b[l] = cmake<C>(Real(0.5) * d.y, Real(-0.5) * d.x);
        }
        const Real kx = (even && 2 * k == nx) ? Real(0) : Real(k) * kfx;
        const long long o = row * g.pxh + k;
        out[0 * g.nc + o] = a[0];
        out[1 * g.nc + o] = b[0];
        out[2 * g.nc + o] = a[1];
        out[5 * g.nc + o] = b[1];
        out[3 * g.nc + o] = cadd(a[2], cmake<C>(kx * b[2].y, -kx * b[2].x));   // Phi_3 - i k_x Phi_V2x
        out[4 * g.nc + o] = cmake<C>(kx * a[3].y, -kx * a[3].x);               // -i k_x Phi_V1x
        out[6 * g.nc + o] = b[3];
        out[7 * g.nc + o] = a[4];
        out[8 * g.nc + o] = b[4];
    }
}

// ------------------------------------------------------------------------------------
// x pass of the second half's start: n_alpha (mixed from slots A and B) -> real space ->
// dPhi/dn_alpha -> half spectra.  grid: ceil(ny nz / LR); 5 lines (component pairs) per row.
// ------------------------------------------------------------------------------------
// NM = 2: the two line-search samples at once (weights from ctl[1] and ctl[2]; the same loads
// of both slots serve both; sample m's nine Phi' spectra go to phi_out + m DFT_NSPEC nc).
template <typename Real, int NX, int NM = 1>
__global__ void __launch_bounds__(kThreads) k_xphi(GridDesc g, AxisPlan px, int LR, const Ctl* __restrict__ ctl,
                                                   const typename Cplx<Real>::type* slotA,
                                                   const typename Cplx<Real>::type* slotB,
                                                   typename Cplx<Real>::type* mat_out,
                                                   typename Cplx<Real>::type* __restrict__ phi_out,
                                                   float* __restrict__ red_max, int* __restrict__ status,
                                                   double* __restrict__ red_phi, Real kfx,
                                                   const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float scratch_f[32];
    __shared__ double scratch_d[32];
    double phi_acc = 0.0;   // sum of Phi(n) over the block's points (grand potential only)
    const int nx = NX > 0 ? NX : g.nx, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    const int lines = 5 * NM * LR;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lines * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long nrows = (long long)g.ny * g.nz;
    const long long row0 = (long long)blockIdx.x * LR;
    Real wA[NM], wB[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const Ctl* cw = NM == 1 ? ctl : ctl + 1 + m;
        wA[m] = CtlW<Real>::wA(cw);
        wB[m] = CtlW<Real>::wB(cw);
    }
    load_wd_rows<Real, NX, NM>(g, LR, row0, nrows, slotA, slotB, wA, wB, mat_out, kfx, A);
    __syncthreads();
    C* R = any_fft<NX, true, false, 0>(A, B, px, lines, 1, pitch, tw);
    float mx = -CUDART_INF_F;
    bool bad = false;
    for (int idx = threadIdx.x; idx < LR * NM * nx; idx += blockDim.x) {
        const int rr = idx / nx, x = idx - (idx / nx) * nx;
        const int r = rr / NM;
        C* base = R + (rr * 5) * pitch + xo<NX>(x);
        Real n[DFT_NCOMP];
        {   // lines (n0, n1), (n2, nV1y), (n3, nV2x), (nV1x, nV1z), (nV2y, nV2z): see wd_comp
            const C v0 = base[0], v1 = base[pitch], v2 = base[2 * pitch], v3 = base[3 * pitch], v4 = base[4 * pitch];
            n[0] = v0.x; n[1] = v0.y; n[2] = v1.x; n[5] = v1.y; n[3] = v2.x;
            n[7] = v2.y; n[4] = v3.x; n[6] = v3.y; n[8] = v4.x; n[9] = v4.y;
        }
        if (row0 + r < nrows) mx = fmaxf(mx, float(n[3]));
        if (red_phi && row0 + r < nrows) phi_acc += phi_value<Real>(n, g.phi);
        const bool ok = phi_derivatives<Real>(n, g.phi);
        if (!ok && row0 + r < nrows) bad = true;
        base[0] = cmake<C>(n[0], n[1]);
        base[pitch] = cmake<C>(n[2], n[5]);
        base[2 * pitch] = cmake<C>(n[3], n[7]);
        base[3 * pitch] = cmake<C>(n[4], n[6]);
        base[4 * pitch] = cmake<C>(n[8], n[9]);
    }
    if (bad) atomicOr(status, DEV_N3BOUND);
    __syncthreads();
    C* other = (R == A) ? B : A;
    C* F = any_fft<NX, false, false, 0>(R, other, px, lines, 1, pitch, tw);
    store_phi_spectra<Real, NX, NM>(g, LR, row0, nrows, kfx, F, phi_out);
    const float bm = block_max(mx, scratch_f);
    if (threadIdx.x == 0 && red_max) red_max[blockIdx.x] = bm;
    if (red_phi) {
        const double bp = block_sum(phi_acc, scratch_d);
        if (threadIdx.x == 0) red_phi[blockIdx.x] = bp;
    }
}

// ------------------------------------------------------------------------------------
// The part of the persistent Phi' x passes after the weighted-density lines of a block's LR rows
// (NM mixtures, the load_wd_rows arrangement) are in A (synced): x C2R, dPhi/dn_alpha at each
// point (the maximum of n3 over the live rows into *mx, n3 >= 1 met into *bad), x R2C, and the
// nine Phi' spectra of each mixture out.  The line buffers stay in use until the caller's next
// barrier.
// ------------------------------------------------------------------------------------
template <typename Real, int NX, int NM>
__device__ __forceinline__ void xphi_rows_ct(const GridDesc& g, int LR, long long row0, long long nrows,
                                             typename Cplx<Real>::type* A, typename Cplx<Real>::type* B,
                                             const typename Cplx<Real>::type* tw, Real kfx,
                                             typename Cplx<Real>::type* __restrict__ phi_out, float* mx,
                                             bool* bad) {
    using C = typename Cplx<Real>::type;
    constexpr int pitch = ct_row_pitch(NX);
    const int lines = 5 * NM * LR;
    C* R = ct_fft<NX, true, false, 0>(A, B, lines, pitch, tw);
    for (int idx = threadIdx.x; idx < LR * NM * NX; idx += kThreads) {
        const int rr = idx / NX, x = idx - (idx / NX) * NX;
        const int r = rr / NM;
        C* bp = R + (rr * 5) * pitch + xo<NX>(x);
        Real n[DFT_NCOMP];
        {   // lines (n0, n1), (n2, nV1y), (n3, nV2x), (nV1x, nV1z), (nV2y, nV2z): see wd_comp
            const C v0 = bp[0], v1 = bp[pitch], v2 = bp[2 * pitch], v3 = bp[3 * pitch], v4 = bp[4 * pitch];
            n[0] = v0.x; n[1] = v0.y; n[2] = v1.x; n[5] = v1.y; n[3] = v2.x;
            n[7] = v2.y; n[4] = v3.x; n[6] = v3.y; n[8] = v4.x; n[9] = v4.y;
        }
        if (row0 + r < nrows) *mx = fmaxf(*mx, float(n[3]));
        const bool okp = phi_derivatives<Real>(n, g.phi);
        if (!okp && row0 + r < nrows) *bad = true;
        bp[0] = cmake<C>(n[0], n[1]);
        bp[pitch] = cmake<C>(n[2], n[5]);
        bp[2 * pitch] = cmake<C>(n[3], n[7]);
        bp[3 * pitch] = cmake<C>(n[4], n[6]);
        bp[4 * pitch] = cmake<C>(n[8], n[9]);
    }
    __syncthreads();
    C* other = (R == A) ? B : A;
    C* F = ct_fft<NX, false, false, 0>(R, other, lines, pitch, tw);
    store_phi_spectra<Real, NX, NM>(g, LR, row0, nrows, kfx, F, phi_out);
}

// ------------------------------------------------------------------------------------
// Persistent form of k_xphi for compile-time lengths (same contract, same arithmetic per block):
// CTA b takes the row blocks b, b + gridDim.x, ...  The nine (one slot) or eighteen (two slots)
// half-spectrum components of a block's LR rows are contiguous in each component, so they
// arrive by one bulk copy each (cp.async.bulk, completing on the stage's mbarrier) into one of
// two staging areas, requested two blocks ahead: the transforms and Phi' of one block run
// while the next blocks' spectra are in flight.  A wait that runs out sets DEV_TIMEOUT and the
// CTA stops after draining the copies it has in flight.
// Shared memory: twiddles | stage 0 | stage 1 (nsrc components of LR rows each) | line
// buffers A, B | two mbarriers.
// ------------------------------------------------------------------------------------
template <typename Real, int NX> __host__ __device__ constexpr size_t xphi_tma_smem(int nm, int LR, int nsrc, int pxh) {
    using C = typename Cplx<Real>::type;
    return (size_t(NX) + 2 * size_t(nsrc) * LR * pxh + 2 * size_t(5 * nm * LR) * ct_row_pitch(NX)) * sizeof(C) +
           2 * sizeof(uint64_t) + 256;
}

template <typename Real, int NX, int NM>
__global__ void __launch_bounds__(kThreads, sizeof(Real) == 4 ? 3 : 1) k_xphi_tma(GridDesc g, int LR, const Ctl* __restrict__ ctl,
                                                       const typename Cplx<Real>::type* slotA,
                                                       const typename Cplx<Real>::type* slotB,
                                                       typename Cplx<Real>::type* mat_out,
                                                       typename Cplx<Real>::type* __restrict__ phi_out,
                                                       float* __restrict__ red_max, int* __restrict__ status,
                                                       Real kfx, const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    static_assert(NX > 0, "compile-time lengths only");
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float scratch_f[32];
    constexpr int pitch = ct_row_pitch(NX);
    const int nsrc = slotB ? 2 * DFT_NSPEC : DFT_NSPEC;
    const int cstride = LR * g.pxh;                       // elements per staged component
    const int lines = 5 * NM * LR;
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127);
    C* tw = reinterpret_cast<C*>(base);
    C* stage0 = tw + ((NX + 15) & ~15);                   // 128-byte aligned (NX a multiple of 16)
    C* A = stage0 + 2 * nsrc * cstride;
    C* B = A + lines * pitch;
    uint64_t* bar = reinterpret_cast<uint64_t*>(B + lines * pitch);
    const long long nrows = (long long)g.ny * g.nz;
    const int nblk = (int)((nrows + LR - 1) / LR);
    Real wA[NM], wB[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const Ctl* cw = NM == 1 ? ctl : ctl + 1 + m;
        wA[m] = CtlW<Real>::wA(cw);
        wB[m] = CtlW<Real>::wB(cw);
    }
    auto issue = [&](int blk, int s) {
        const long long r0 = (long long)blk * LR;
        const int rows = (int)(nrows - r0 < LR ? nrows - r0 : LR);
        const uint32_t bytes = uint32_t(rows) * uint32_t(g.pxh) * uint32_t(sizeof(C));
        C* st = stage0 + s * nsrc * cstride;
        tma::mbar_expect_tx(&bar[s], bytes * uint32_t(nsrc));
        for (int c = 0; c < nsrc; ++c) {
            const C* src = (c < DFT_NSPEC ? slotA + (long long)c * g.nc : slotB + (long long)(c - DFT_NSPEC) * g.nc) +
                           r0 * g.pxh;
            tma::bulk_load(st + c * cstride, src, bytes, &bar[s]);
        }
    };
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = twx[i];
    __syncthreads();
    int issued = 0, consumed = 0;   // per stage, packed (stage 1 << 16) | stage 0; thread 0
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            const int blk = blockIdx.x + s * gridDim.x;
            if (blk < nblk) { issue(blk, s); issued += 1 << (16 * s); }
        }
    }
    bool bad = false;
    int it = 0;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x, ++it) {
        const int cur = it & 1;
        const long long row0 = (long long)blk * LR;
        const bool ok = tma::mbar_wait(&bar[cur], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, DEV_TIMEOUT);
                for (int s = 0; s < 2; ++s) {
                    const int n_is = (issued >> (16 * s)) & 0xffff, n_co = (consumed >> (16 * s)) & 0xffff;
                    if (n_is > n_co) tma::mbar_wait(&bar[s], (n_is - 1) & 1);
                }
            }
            break;
        }
        consumed += 1 << (16 * cur);
        const C* st = stage0 + cur * nsrc * cstride;
        load_wd_rows<Real, NX, NM, true>(g, LR, row0, nrows, nullptr, slotB, wA, wB, mat_out, kfx, A, st, cstride);
        __syncthreads();
        // the stage is free: request the block after next into it while this one is transformed
        if (threadIdx.x == 0) {
            const int next = blk + 2 * gridDim.x;
            if (next < nblk) { issue(next, cur); issued += 1 << (16 * cur); }
        }
        float mx = -CUDART_INF_F;
        xphi_rows_ct<Real, NX, NM>(g, LR, row0, nrows, A, B, tw, kfx, phi_out, &mx, &bad);
        const float bm = block_max(mx, scratch_f);
        if (threadIdx.x == 0 && red_max) red_max[blk] = bm;
        __syncthreads();   // the line buffers are rewritten by the next block
    }
    if (bad) atomicOr(status, DEV_N3BOUND);
}

// ------------------------------------------------------------------------------------
// Persistent form of k_xphi with one staging area filled by per-thread 16-byte asynchronous
// copies (cp.async; same contract, same arithmetic per block): the spectra of a CTA's next row
// block are requested as soon as the current block's have been turned into lines, and arrive
// while it is transformed.  Each thread waits for its own copies, then a barrier: no mbarrier,
// no bound needed.  Shared memory: twiddles | stage (nsrc components of LR rows) | line buffers
// A, B.  Row blocks of a component are contiguous and start on 16-byte boundaries (pxh even).
// ------------------------------------------------------------------------------------
template <typename Real, int NX> __host__ __device__ constexpr size_t xphi_cpa_smem(int nm, int LR, int nsrc, int pxh) {
    using C = typename Cplx<Real>::type;
    return (size_t(NX) + size_t(nsrc) * LR * pxh + 2 * size_t(5 * nm * LR) * ct_row_pitch(NX)) * sizeof(C) + 128;
}

template <typename Real, int NX, int NM>
__global__ void __launch_bounds__(kThreads, sizeof(Real) == 4 ? 3 : 1) k_xphi_cpa(GridDesc g, int LR, const Ctl* __restrict__ ctl,
                                                       const typename Cplx<Real>::type* slotA,
                                                       const typename Cplx<Real>::type* slotB,
                                                       typename Cplx<Real>::type* mat_out,
                                                       typename Cplx<Real>::type* __restrict__ phi_out,
                                                       float* __restrict__ red_max, int* __restrict__ status,
                                                       Real kfx, const typename Cplx<Real>::type* __restrict__ twx) {
    static_assert(NX > 0, "compile-time lengths only");
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float scratch_f[32];
    const int nsrc = slotB ? 2 * DFT_NSPEC : DFT_NSPEC;
    const int cstride = LR * g.pxh;                       // elements per staged component
    const int lines = 5 * NM * LR;
    constexpr int pitch = ct_row_pitch(NX);
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127);
    C* tw = reinterpret_cast<C*>(base);
    C* stage = tw + ((NX + 15) & ~15);                    // 128-byte aligned (NX a multiple of 16)
    C* A = stage + nsrc * cstride;
    C* B = A + lines * pitch;
    const long long nrows = (long long)g.ny * g.nz;
    const int nblk = (int)((nrows + LR - 1) / LR);
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = twx[i];
    dep_launch();
    dep_wait();
    Real wA[NM], wB[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const Ctl* cw = NM == 1 ? ctl : ctl + 1 + m;
        wA[m] = CtlW<Real>::wA(cw);
        wB[m] = CtlW<Real>::wB(cw);
    }
    // the nsrc components of row block blk, in 16-byte chunks spread over the threads
    auto issue = [&](int blk) {
        const long long r0 = (long long)blk * LR;
        const int rows = (int)(nrows - r0 < LR ? nrows - r0 : LR);
        const int per = int((long long)rows * g.pxh * sizeof(C) / 16);
        for (int i = threadIdx.x; i < nsrc * per; i += kThreads) {
            const int c = i / per, q = i - c * per;
            const C* src = (c < DFT_NSPEC ? slotA + (long long)c * g.nc : slotB + (long long)(c - DFT_NSPEC) * g.nc) +
                           r0 * g.pxh;
            tma::cp16(reinterpret_cast<char*>(stage + c * cstride) + 16 * q, reinterpret_cast<const char*>(src) + 16 * q);
        }
        tma::cp_commit();
    };
    if (blockIdx.x < nblk) issue(blockIdx.x);
    bool bad = false;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long row0 = (long long)blk * LR;
        tma::cp_wait_all();
        __syncthreads();
        load_wd_rows<Real, NX, NM, true>(g, LR, row0, nrows, nullptr, slotB, wA, wB, mat_out, kfx, A, stage, cstride);
        __syncthreads();
        // the stage is free: request the next block into it while this one is transformed
        if (blk + gridDim.x < nblk) issue(blk + gridDim.x);
        float mx = -CUDART_INF_F;
        xphi_rows_ct<Real, NX, NM>(g, LR, row0, nrows, A, B, tw, kfx, phi_out, &mx, &bad);
        const float bm = block_max(mx, scratch_f);
        if (threadIdx.x == 0 && red_max) red_max[blk] = bm;
        __syncthreads();   // the line buffers are rewritten by the next block
    }
    if (bad) atomicOr(status, DEV_N3BOUND);
}

// ------------------------------------------------------------------------------------
// z pass of the second half.  grid (ceil(nxh/T), ny)
//   phi:  in  10 dPhi/dn_alpha spectra after x, y forward (kx, ky, z)
//         out S one-body correlation spectra after z inverse, 1/N applied (kx, ky, z)
//   mu_hat_i = sum_alpha Phi_hat_alpha w_hat_i^alpha(+k) (eq. muHS): with the vector weights
//   w_hat^V2 = -i k w_hat^3 and w_hat^V1 = w_hat^V2/(4 pi R) the k-space sum needs only the five
//   species-independent spectra Phi0, Phi1, Phi2, Phi3 + div(PhiV2), div(PhiV1).
//   c_hat_i = (-mu_hat_i + wA es_A_i + wB es_B_i) / N.
// flags: 1 = hard-sphere part, 2 = electrostatic part; ncomp_out = S (or S + 1 for psi).
// ------------------------------------------------------------------------------------
template <typename Real, int NZ, int TZ>
__global__ void __launch_bounds__(kThreads) k_zconv_bwd(GridDesc g, AxisPlan pz, SpeciesDesc<Real> sp, int Trt,
                                                        Real kfx, Real kfy, Real kfz, int flags, int ncomp_out,
                                                        const Ctl* __restrict__ ctl,
                                                        typename Cplx<Real>::type* phi,
                                                        const typename Cplx<Real>::type* esA,
                                                        const typename Cplx<Real>::type* esB,
                                                        typename Cplx<Real>::type* es_mat,
                                                        const typename Cplx<Real>::type* __restrict__ twz) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    const int nz = NZ > 0 ? NZ : g.nz, ny = g.ny, nxh = g.nxh, S = sp.S;
    const int T = TZ > 0 ? TZ : Trt;
    const int tile = T * nz;
    C* tw = align_ptr<C>(smem_raw);
    C* pool[7];
    for (int i = 0; i < 7; ++i) pool[i] = tw + nz + i * tile;
    for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = twz[i];
    const int kx0 = blockIdx.x * T;
    const int kyi = blockIdx.y;
    const long long zstride = (long long)ny * g.pxh;
    const long long col0 = (long long)kyi * g.pxh + kx0;
    const bool hs = (flags & 1) != 0, es_on = (flags & 2) != 0;
    const Real wA = CtlW<Real>::wA(ctl), wB = CtlW<Real>::wB(ctl);

    if (hs) {
        // nine Phi' spectra (DFT_NSPEC order): 0..3 transform into accumulators 0..3, B4 into
        // accumulator 4; -i k_y / -i k_z of Phi_V1y, Phi_V1z add to accumulator 4 and of Phi_V2y,
        // Phi_V2z to accumulator 3 (Nyquist components of their axis dropped)
        for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) pool[4][idx] = cmake<C>(Real(0), Real(0));
        for (int a = 0; a < DFT_NSPEC; ++a) {
            C* dst = (a < 4) ? pool[a] : pool[5];
            tile_load<TZ, NZ>(dst, phi + (long long)a * g.nc + col0, zstride, nxh - kx0, T, nz);
            __syncthreads();
            C* r = any_fft<NZ, false, true, TZ>(dst, pool[6], pz, T, T, 1, tw);
            if (a < 4) {
                if (r != dst) { pool[6] = dst; pool[a] = r; }
                continue;
            }
            C* acc = (a < 7) ? pool[4] : pool[3];
            const int d = (a == 4) ? 0 : ((a == 5 || a == 7) ? 1 : 2);
            for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
                const int kzi = idx / T;
                const C u = r[idx];
                if (d == 0) { acc[idx] = cadd(acc[idx], u); continue; }
                Real kd;
                bool nyq;
                if (d == 1) { kd = kval<Real>(kyi, g.ny, kfy); nyq = (g.ny % 2 == 0) && (2 * kyi == g.ny); }
                else { kd = kval<Real>(kzi, g.nz, kfz); nyq = (g.nz % 2 == 0) && (2 * kzi == g.nz); }
                if (!nyq) acc[idx] = cadd(acc[idx], cmake<C>(kd * u.y, -kd * u.x));    // -i k_d u
            }
            __syncthreads();
        }
    }

    const Real fourpi = Real(4.0 * CUDART_PI);
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int kzi = idx / T, t = idx - (idx / T) * T;
        const int kxi = kx0 + t;
        C out[DFT_MAXS + 1];
        for (int s = 0; s < DFT_MAXS + 1; ++s) out[s] = cmake<C>(Real(0), Real(0));
        if (hs) {
            const KPoint<Real> p = kpoint<Real>(g, kxi, kyi, kzi, kfx, kfy, kfz);
            const C a0 = pool[0][idx], a1 = pool[1][idx], a2 = pool[2][idx], a3 = pool[3][idx], a4 = pool[4][idx];
            for (int s = 0; s < S; ++s) {
                Real w0, j3;
                const Real R = sp.R[s];
                fmt_weights<Real>(p.kmag, R, &w0, &j3);
                C mu = cscale(a0, w0);
                mu = cadd(mu, cscale(a1, R * w0));
                mu = cadd(mu, cscale(a2, fourpi * R * R * w0));
                mu = cadd(mu, cscale(a3, fourpi * R * R * R * j3));
                mu = cadd(mu, cscale(a4, R * R * j3));
                out[s] = cmake<C>(-mu.x, -mu.y);
            }
        }
        if (es_on && kxi < nxh) {
            const long long o = (long long)kzi * zstride + col0 + t;
            for (int s = 0; s < ncomp_out; ++s) {
                C e = cscale(esA[(long long)s * g.nc + o], wA);
                if (esB) e = cadd(e, cscale(esB[(long long)s * g.nc + o], wB));
                if (es_mat) es_mat[(long long)s * g.nc + o] = e;
                out[s] = cadd(out[s], e);
            }
        }
        for (int s = 0; s < ncomp_out; ++s) pool[s][idx] = cscale(out[s], sp.inv_n);
    }
    __syncthreads();

    for (int s = 0; s < ncomp_out; ++s) {
        C* r = any_fft<NZ, true, true, TZ>(pool[s], pool[5 + (s & 1)], pz, T, T, 1, tw);
        tile_store<TZ, NZ>(phi + (long long)s * g.nc + col0, r, zstride, nxh - kx0, T, nz);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Normalisation of fixed-number species: per block, sum over accessible points of
// e_i = exp(-V_i + c_i) for the species with canon[i] (c_i from the half spectra cspec),
// red[block * DFT_MAXS + i].  Only the complex lines holding such species are transformed.
// grid: ceil(ny nz / LR); nl lines per row (line l = species pair (2 line_of[l], +1)).
// ------------------------------------------------------------------------------------
template <typename Real, int NX>
__global__ void __launch_bounds__(kThreads) k_xcanon(GridDesc g, AxisPlan px, SpeciesDesc<Real> sp, int LR, int nl,
                                                     int line0, int line1, int line2,
                                                     const typename Cplx<Real>::type* __restrict__ cspec,
                                                     const Real* __restrict__ V, double* __restrict__ red,
                                                     const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double scratch_d[32];
    const int nx = NX > 0 ? NX : g.nx, nxh = nx / 2 + 1, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1, S = sp.S;
    const bool even = (nx % 2) == 0;
    const int lines = nl * LR;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lines * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long nrows = (long long)g.ny * g.nz;
    const long long row0 = (long long)blockIdx.x * LR;
    const int line_of[3] = {line0, line1, line2};
    for (int idx = threadIdx.x; idx < lines * nxh; idx += blockDim.x) {
        const int l = idx / nxh, k = idx - (idx / nxh) * nxh;
        const int r = l / nl, j = l - (l / nl) * nl;
        const long long row = row0 + r;
        const int ca = 2 * line_of[j], cb = ca + 1;
        C a = cmake<C>(Real(0), Real(0)), b = a;
        if (row < nrows) {
            a = cspec[(long long)ca * g.nc + row * g.pxh + k];
            if (cb < S) b = cspec[(long long)cb * g.nc + row * g.pxh + k];
        }
        const bool edge = k == 0 || (even && 2 * k == nx);
        if (edge) { a.y = Real(0); b.y = Real(0); }
        A[l * pitch + xo<NX>(k)] = cmake<C>(a.x - b.y, a.y + b.x);
        if (!edge) A[l * pitch + xo<NX>(nx - k)] = cmake<C>(a.x + b.y, b.x - a.y);
    }
    __syncthreads();
    C* R = any_fft<NX, true, false, 0>(A, B, px, lines, 1, pitch, tw);
    Real acc[DFT_MAXS], comp[DFT_MAXS];
#pragma unroll
    for (int s = 0; s < DFT_MAXS; ++s) acc[s] = comp[s] = Real(0);
    for (int idx = threadIdx.x; idx < LR * nx; idx += blockDim.x) {
        const int r = idx / nx, x = idx - (idx / nx) * nx;
        const long long row = row0 + r;
        if (row >= nrows) continue;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= nl) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int s = 2 * line_of[j] + h;
                if (s >= S || !sp.canon[s]) continue;
                const C pr = R[(r * nl + j) * pitch + xo<NX>(x)];
                const Real c = h ? pr.y : pr.x;
                const Real v = V[(long long)s * g.n + row * nx + x];
                const Real e = (isinf(v) && v > Real(0)) ? Real(0) : exp(-v + c);
#pragma unroll
                for (int q = 0; q < DFT_MAXS; ++q) {
                    if (q != s) continue;
                    const Real y = e - comp[q];
                    const Real t = acc[q] + y;
                    comp[q] = (t - acc[q]) - y;
                    acc[q] = t;
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < DFT_MAXS; ++s) {
        if (s >= S || !sp.canon[s]) continue;      // uniform across the block
        double bs;
        if constexpr (sizeof(Real) == 4) bs = block_sum_ds(acc[s], -comp[s], scratch_d);
        else bs = block_sum(double(acc[s]) - double(comp[s]), scratch_d);
        if (threadIdx.x == 0) red[(long long)blockIdx.x * DFT_MAXS + s] = bs;
    }
}

// canon_scale_i = (N_i / h^3) / sum over blocks of the k_xcanon partial sums (one block).
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_canon_scale(Ctl* ctl, SpeciesDesc<Real> sp, const double* __restrict__ red,
                                                          int nblocks) {
    dep_launch();
    dep_wait();
    __shared__ double scratch_d[32];
    for (int s = 0; s < sp.S; ++s) {
        if (!sp.canon[s]) continue;
        double t = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += red[(long long)b * DFT_MAXS + s];
        const double tot = block_sum(t, scratch_d);
        if (threadIdx.x == 0) {
            ctl->canon_scale[s] = sp.nfix_dv[s] / tot;
            if (!(tot > 0.0) || !isfinite(tot)) ctl->status |= DEV_NONFINITE;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Final x pass: one-body correlations c_i (half spectra) -> real space -> Picard map
//   G_i = rho_bath_i exp(beta mu_HS_bath_i - V_i + c_i)   (0 where V_i = +inf)
// at rho = w0 rho0 + w1 rho1, with the residual sum_i sum_x ((rho_i - G_i)/rho_bath_i)^2
// accumulated in FP64.  grid: ceil(ny nz / LR); ceil(S/2) lines per row.
// rho_out may alias rho0 and g_out may alias rho1 (each point is read before it is written).
// ------------------------------------------------------------------------------------
// NM = 2: the two line-search samples at once -- the c spectra of sample m at cspec (m = 0) and
// cspec2 (m = 1), weights from ctl[1 + m], rho0, rho1, V (and the low part) read once for both;
// the residual sums of sample m go to red_sum / red_sum2; nothing is written to rho or G.
template <typename Real, int NX, int NM = 1>
__global__ void __launch_bounds__(kThreads, sizeof(Real) == 4 ? 3 : 2) k_xupdate(GridDesc g, AxisPlan px, SpeciesDesc<Real> sp, int LR,
                                                      const Ctl* __restrict__ ctl,
                                                      const typename Cplx<Real>::type* __restrict__ cspec,
                                                      const typename Cplx<Real>::type* __restrict__ cspec2,
                                                      const Real* rho0, const Real* rho1,
                                                      const Real* __restrict__ V, Real* rho_out, Real* g_out,
                                                      typename Cplx<Real>::type* __restrict__ gspec_out,
                                                      Real* rho_lo, double* __restrict__ red_sum,
                                                      double* __restrict__ red_sum2, int* __restrict__ status,
                                                      const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double scratch_d[32];
    const int nx = NX > 0 ? NX : g.nx, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1, S = sp.S;
    const int lpr = (S + 1) / 2;
    const int lines = NM * lpr * LR;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lines * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long nrows = (long long)g.ny * g.nz;
    const long long row0 = (long long)blockIdx.x * LR;
    load_species_rows<Real, NX, NM>(g, LR, row0, nrows, S, cspec, cspec2, A);
    const int total = LR * nx;
    // G_i = pref_i exp(mu0_i - V_i + c_i): the bath (rho_b, beta mu_HS,b), or for a
    // fixed-number species the normalisation of this evaluation and no bath constant
    __shared__ Real s_pref[DFT_MAXS], s_mu0[DFT_MAXS], s_irb[DFT_MAXS];
    if (threadIdx.x < DFT_MAXS) {
        const int s = threadIdx.x;
        const bool cn = s < S && sp.canon[s];
        s_pref[s] = cn ? Real(ctl->canon_scale[s]) : sp.rho_b[s];
        s_mu0[s] = cn ? Real(0) : sp.mu_hs_b[s];
        s_irb[s] = sp.inv_rho_b[s];
    }
    __syncthreads();
    C* R = any_fft<NX, true, false, 0>(A, B, px, lines, 1, pitch, tw);
    Real w0[NM], w1[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const Ctl* cw = NM == 1 ? ctl : ctl + 1 + m;
        w0[m] = CtlW<Real>::w0(cw);
        w1[m] = CtlW<Real>::w1(cw);
    }
    // per-thread partial sums in the working precision with Kahan compensation, then
    // double-single (FP32) or FP64 across threads, FP64 across blocks
    Real acc[NM], comp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = comp[m] = Real(0);
    bool bad = false;
    // one point of species s under mixture m: new iterate (and its low part), G, squared
    // weighted residual
    auto point = [&](int m, int s, Real c, Real r0, Real r1, Real v, Real l0, Real& rho, Real& lo, Real& gval) {
        lo = Real(0);
        if (rho_lo) {
            // extended iterate rho0 = r0 + l0 (a value and its rounding error):
            // rho = rho0 + w1 (rho1 - rho0) formed so that steps below half an ulp of rho0
            // accumulate in the low part instead of rounding away (w0 = 1 - w1), then split
            // again into rho + lo by an error-free sum (Knuth's TwoSum)
            const Real t = l0 + w1[m] * ((r1 - r0) - l0);
            rho = r0 + t;
            const Real bv = rho - r0;
            lo = (r0 - (rho - bv)) + (t - bv);
        } else {
            rho = w0[m] * r0 + w1[m] * r1;
        }
        if (isinf(v) && v > Real(0)) gval = Real(0);
        else gval = s_pref[s] * exp(s_mu0[s] - v + c);
        if (!isfinite(gval) || !isfinite(rho)) bad = true;
        const Real d = ((rho - gval) + lo) * s_irb[s];
        const Real y = d * d - comp[m];
        const Real t = acc[m] + y;
        comp[m] = (t - acc[m]) - y;
        acc[m] = t;
    };
    // rho_out / g_out / rho_lo may alias rho0 / rho1 / the low part read: every value is read
    // before the same thread writes that element, and the threads' elements are distinct
    if constexpr (NX > 0) {
        // compile-time lengths: items (species, group of VW consecutive points of a row),
        // KB items per thread with their 16-byte loads of rho0, rho1, V (and the low part)
        // issued before any is used, results stored 16 bytes at a time
        using V16 = typename Vec16<Real>::type;
        constexpr int VW = Vec16<Real>::n;
        constexpr int KB = DFT_XUPD_BATCH;
        static_assert(NX % VW == 0, "row length a multiple of the vector width");
        const int groups = total / VW;
        const int items = S * groups;
        // item it = s groups + gi, kept as (s, gi) and advanced without dividing
        int s_b = threadIdx.x / groups, gi_b = threadIdx.x - s_b * groups;
        for (int base = threadIdx.x; base < items; base += KB * kThreads) {
            V16 a0[KB], a1[KB], av[KB], al[KB];
            int sj[KB], gj[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                if (j == 0) { sj[0] = s_b; gj[0] = gi_b; }
                else {
                    sj[j] = sj[j - 1];
                    gj[j] = gj[j - 1] + kThreads;
                    while (gj[j] >= groups) { gj[j] -= groups; ++sj[j]; }
                }
                const int it = base + j * kThreads;
                const int s = sj[j], gi = gj[j];
                const bool live = it < items && row0 + (gi * VW) / NX < nrows;
                const long long o = (long long)s * g.n + row0 * NX + (long long)gi * VW;
                a0[j] = a1[j] = av[j] = al[j] = vzero<V16>();
                if (live) {
                    a0[j] = ld16(rho0 + o);
                    if (rho1) a1[j] = ld16(rho1 + o);
                    av[j] = ld16(V + o);
                    if (rho_lo) al[j] = ld16(rho_lo + o);
                }
            }
            gi_b += KB * kThreads;
            while (gi_b >= groups) { gi_b -= groups; ++s_b; }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                const int it = base + j * kThreads;
                const int s = sj[j], gi = gj[j];
                const int idx = gi * VW, r = idx / NX, x = idx - (idx / NX) * NX;
                if (!(it < items && row0 + r < nrows)) continue;
                const long long o = (long long)s * g.n + row0 * NX + idx;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    C* Rl = R + (m * lpr * LR + r * lpr + s / 2) * pitch;
                    V16 orho, og, olo;
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        // this species' half of the line (the other species of the line is another
                        // item's); with gspec_out, G goes back into the same half
                        Real* hp = reinterpret_cast<Real*>(Rl + xo<NX>(x + e)) + (s & 1);
                        point(m, s, *hp, vel(a0[j], e), vel(a1[j], e), vel(av[j], e), vel(al[j], e), vel(orho, e),
                              vel(olo, e), vel(og, e));
                        if (NM == 1 && gspec_out) *hp = vel(og, e);
                    }
                    if (NM == 1 && rho_out) {
                        st16(rho_out + o, orho);
                        if (rho_lo) st16(rho_lo + o, olo);
                    }
                    if (NM == 1 && g_out) st16(g_out + o, og);
                }
            }
        }
    } else {
        // run-time lengths: one point per thread at a time, its rho0, rho1, V (and low part)
        // loaded one point ahead of their use
        Real r0[DFT_MAXS], r1[DFT_MAXS], vv[DFT_MAXS], rl[DFT_MAXS];
        auto load_point = [&](int idx, Real* a0, Real* a1, Real* av, Real* al) {
            const long long row = row0 + idx / nx;
            const bool live = idx < total && row < nrows;
            const long long pt = row0 * nx + idx;
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                a0[s] = a1[s] = av[s] = al[s] = Real(0);
                if (s < S && live) {
                    const long long o = (long long)s * g.n + pt;
                    a0[s] = rho0[o];
                    a1[s] = rho1 ? rho1[o] : Real(0);
                    av[s] = V[o];
                    if (rho_lo) al[s] = rho_lo[o];
                }
            }
        };
        load_point(threadIdx.x, r0, r1, vv, rl);
        for (int idx = threadIdx.x; idx < total; idx += kThreads) {
            Real n0[DFT_MAXS], n1[DFT_MAXS], nv[DFT_MAXS], nl[DFT_MAXS];
            load_point(idx + kThreads, n0, n1, nv, nl);
            const int r = idx / nx, x = idx - (idx / nx) * nx;
            if (row0 + r < nrows) {
                const long long pt = row0 * nx + idx;
#pragma unroll
                for (int s = 0; s < DFT_MAXS; ++s) {
                    if (s >= S) continue;
                    const long long o = (long long)s * g.n + pt;
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        Real* hp = reinterpret_cast<Real*>(R + (m * lpr * LR + r * lpr + s / 2) * pitch + xo<NX>(x)) +
                                   (s & 1);
                        Real rho, lo, gval;
                        point(m, s, *hp, r0[s], r1[s], vv[s], rl[s], rho, lo, gval);
                        if (NM == 1 && gspec_out) *hp = gval;
                        if (NM == 1 && rho_out) {
                            rho_out[o] = rho;
                            if (rho_lo) rho_lo[o] = lo;
                        }
                        if (NM == 1 && g_out) g_out[o] = gval;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < DFT_MAXS; ++s) {
                r0[s] = n0[s];
                r1[s] = n1[s];
                vv[s] = nv[s];
                rl[s] = nl[s];
            }
        }
    }
    if (bad) atomicOr(status, DEV_NONFINITE);
    if (NM == 1 && gspec_out) {
        // the x half spectra of the G rows just formed (the next first half's input): the lines
        // now hold G in place of c1, two species per complex line
        __syncthreads();
        C* other = (R == A) ? B : A;
        C* F = any_fft<NX, false, false, 0>(R, other, px, lines, 1, pitch, tw);
        store_pair_rows<Real, NX>(g, lines, lpr, row0, nrows, S, F, gspec_out);
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        double bs;
        if constexpr (sizeof(Real) == 4) bs = block_sum_ds(acc[m], -comp[m], scratch_d);
        else bs = block_sum(double(acc[m]) - double(comp[m]), scratch_d);
        if (threadIdx.x == 0) (m == 0 ? red_sum : red_sum2)[blockIdx.x] = bs;
    }
}

// ------------------------------------------------------------------------------------
// Gradient pass: x inverse of the one-body correlations c_i, then at each point
//   dOmega/drho_i = h^3 [ln(rho_i / rho_bath_i) + V_i - beta mu_HS_bath_i - c_i]   (accessible, rho > 0)
//   dOmega/dV_i   = h^3 rho_i
// and per-block sums red[b (S + 1) + 0] = sum_i sum_x [rho_i (ln(rho_i/rho_bath_i) - 1) + rho_i (V_i -
// beta mu_ex_bath_i)] (accessible points), red[b (S + 1) + 1 + i] = sum_x rho_i, all in FP64.
// ------------------------------------------------------------------------------------
template <typename Real, int NX>
__global__ void __launch_bounds__(kThreads) k_xgrad(GridDesc g, AxisPlan px, SpeciesDesc<Real> sp, int LR, Real dv,
                                                    const typename Cplx<Real>::type* __restrict__ cspec,
                                                    const Real* __restrict__ rho, const Real* __restrict__ V,
                                                    Real* __restrict__ grad_rho, Real* __restrict__ grad_V,
                                                    double* __restrict__ red,
                                                    const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double scratch_d[32];
    const int nx = NX > 0 ? NX : g.nx, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1, S = sp.S;
    const int lpr = (S + 1) / 2;
    const int lines = lpr * LR;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lines * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long nrows = (long long)g.ny * g.nz;
    const long long row0 = (long long)blockIdx.x * LR;
    load_pair_rows<Real, NX>(g, lines, lpr, row0, nrows, S, cspec, nullptr, Real(1), Real(0), nullptr, A);
    __syncthreads();
    C* R = any_fft<NX, true, false, 0>(A, B, px, lines, 1, pitch, tw);
    double acc[DFT_MAXS + 1];
    for (int s = 0; s <= DFT_MAXS; ++s) acc[s] = 0.0;
    for (int idx = threadIdx.x; idx < LR * nx; idx += blockDim.x) {
        const int r = idx / nx, x = idx - (idx / nx) * nx;
        const long long row = row0 + r;
        if (row >= nrows) continue;
        for (int s = 0; s < S; ++s) {
            const C pr = R[(r * lpr + s / 2) * pitch + xo<NX>(x)];
            const Real c = (s & 1) ? pr.y : pr.x;
            const long long o = (long long)s * g.n + row * nx + x;
            const Real rv = rho[o];
            const Real v = V[o];
            const bool acc_ok = !(isinf(v) && v > Real(0)) && rv > Real(0);
            Real gr = Real(0);
            if (acc_ok) {
                const double lr = log(double(rv) * double(sp.inv_rho_b[s]));
                gr = Real(dv * (lr + double(v) - double(sp.mu_hs_b[s]) - double(c)));
                acc[0] += double(rv) * (lr - 1.0) + double(rv) * (double(v) - double(sp.mu_ex_b[s]));
            }
            acc[1 + s] += double(rv);
            if (grad_rho) grad_rho[o] = gr;
            if (grad_V) grad_V[o] = dv * rv;
        }
    }
    for (int s = 0; s <= S; ++s) {
        const double b = block_sum(acc[s], scratch_d);
        if (threadIdx.x == 0) red[(long long)blockIdx.x * (S + 1) + s] = b;
    }
}

// ------------------------------------------------------------------------------------
// Plain x inverse of ncomp half spectra to real fields, out[c] = value + offset[c].
// Optional max of component cmax into red_max.  grid: ceil(ny nz / LR).
// ------------------------------------------------------------------------------------
template <typename Real, int NX>
__global__ void __launch_bounds__(kThreads) k_xinv(GridDesc g, AxisPlan px, int LR, int ncomp,
                                                   const typename Cplx<Real>::type* __restrict__ spec,
                                                   Real* __restrict__ out, Real* __restrict__ out_last,
                                                   Offsets<Real> off, int cmax,
                                                   float* __restrict__ red_max, int wd, Real kfx,
                                                   const typename Cplx<Real>::type* __restrict__ twx) {
    dep_launch();
    dep_wait();
    using C = typename Cplx<Real>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float scratch_f[32];
    const int nx = NX > 0 ? NX : g.nx, pitch = NX > 0 ? ct_row_pitch(NX) : nx + 1;
    // one component without outputs (the maximum only): two grid rows per complex line
    const bool rows2 = ncomp == 1 && !wd && !out && !out_last;
    const int lpr = (ncomp + 1) / 2;
    const int lines = rows2 ? (LR + 1) / 2 : lpr * LR;
    C* tw = align_ptr<C>(smem_raw);
    C* A = tw + nx;
    C* B = A + lines * pitch;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = twx[i];
    const long long nrows = (long long)g.ny * g.nz;
    const long long row0 = (long long)blockIdx.x * LR;
    const Real one = Real(1), zero = Real(0);
    if (wd) load_wd_rows<Real, NX>(g, LR, row0, nrows, spec, nullptr, &one, &zero, nullptr, kfx, A);
    else if (rows2) load_row_pairs<Real, NX>(g, LR, row0, nrows, spec, A);
    else load_pair_rows<Real, NX>(g, lines, lpr, row0, nrows, ncomp, spec, nullptr, Real(1), Real(0), nullptr, A);
    __syncthreads();
    C* R = any_fft<NX, true, false, 0>(A, B, px, lines, 1, pitch, tw);
    float mx = -CUDART_INF_F;
    for (int idx = threadIdx.x; idx < LR * nx; idx += blockDim.x) {
        const int r = idx / nx, x = idx - (idx / nx) * nx;
        const long long row = row0 + r;
        if (row >= nrows) continue;
        if (rows2) {
            const C pr = R[(r / 2) * pitch + xo<NX>(x)];
            mx = fmaxf(mx, float(((r & 1) ? pr.y : pr.x) + off.v[0]));
            continue;
        }
        for (int c = 0; c < ncomp; ++c) {
            const int l = wd ? wd_line(c) : c / 2, j = wd ? wd_slot(c) : (c & 1);
            const C pr = R[(r * lpr + l) * pitch + xo<NX>(x)];
            const Real v = (j ? pr.y : pr.x) + off.v[c];
            if (out_last && c == ncomp - 1) out_last[row * nx + x] = v;
            else if (out) out[(long long)c * g.n + row * nx + x] = v;
            if (c == cmax) mx = fmaxf(mx, float(v));
        }
    }
    if (red_max) {
        const float bm = block_max(mx, scratch_f);
        if (threadIdx.x == 0) red_max[blockIdx.x] = bm;
    }
}

#ifdef DFT_DEFINE_FINALIZE
// ------------------------------------------------------------------------------------
// Line-search bookkeeping on the device (Sec. "Nonlinear solver"), one block.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void set_weights(Ctl* c, double a) {
    c->wA = 1.0 - a; c->wB = a; c->w0 = 1.0 - a; c->w1 = a;
    c->wAf = float(c->wA); c->wBf = float(c->wB); c->w0f = float(c->w0); c->w1f = float(c->w1);
}

// ctl points at three control blocks: the iteration's, then the weights of the two line-search
// samples (ctl[1], ctl[2]: wA, wB, w0, w1 only), which FIN_AMAX sets for the paired evaluation.
template <int B>
__device__ __forceinline__ double partial_sum(const double* __restrict__ red_sum, int nsum) {
    // four independent partial results per thread, so that a thread's loads are all in flight
    // at once (the partial sums are L2-resident: the kernel is a few load latencies long)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * B < nsum; i += 4 * B) {
        s0 += red_sum[i];
        s1 += red_sum[i + B];
        s2 += red_sum[i + 2 * B];
        s3 += red_sum[i + 3 * B];
    }
    for (; i < nsum; i += B) s0 += red_sum[i];
    return (s0 + s1) + (s2 + s3);
}

template <int B>
__global__ void __launch_bounds__(B) k_finalize(Ctl* ctl, const double* __restrict__ red_sum,
                                                          const double* __restrict__ red_sum2, int nsum,
                                                          const float* __restrict__ red_max, int nmax, int op,
                                                          double inv_count, double alpha_fixed, double n3_bound,
                                                          double alpha_floor) {
    dep_launch();
    dep_wait();
    __shared__ double scratch_d[64];
    __shared__ float scratch_f[32];
    double s = partial_sum<B>(red_sum, nsum);
    double s_2 = red_sum2 ? partial_sum<B>(red_sum2, nsum) : 0.0;
    float m0 = -CUDART_INF_F, m1 = -CUDART_INF_F, m2 = -CUDART_INF_F, m3 = -CUDART_INF_F;
    int i = threadIdx.x;
    for (; i + 3 * B < nmax; i += 4 * B) {
        m0 = fmaxf(m0, red_max[i]);
        m1 = fmaxf(m1, red_max[i + B]);
        m2 = fmaxf(m2, red_max[i + 2 * B]);
        m3 = fmaxf(m3, red_max[i + 3 * B]);
    }
    for (; i < nmax; i += B) m0 = fmaxf(m0, red_max[i]);
    float m = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
    // the two sums and the maximum through one pair of barriers (the same order of operations
    // per quantity as block_sum / block_max)
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s_2 += __shfl_xor_sync(0xffffffffu, s_2, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) { scratch_d[w] = s; scratch_d[32 + w] = s_2; scratch_f[w] = m; }
        __syncthreads();
        if (threadIdx.x >= 32) return;
        const bool in = l < B / 32;
        s = in ? scratch_d[l] : 0.0;
        s_2 = in ? scratch_d[32 + l] : 0.0;
        m = in ? scratch_f[l] : -CUDART_INF_F;
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            s_2 += __shfl_xor_sync(0xffffffffu, s_2, o);
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
    }
    const double tot = s, tot2 = s_2;
    const float mx = m;
    if (threadIdx.x != 0) return;
    Ctl* c = ctl;
    const double f = tot * inv_count;
    if (op & FIN_IDENTITY) {
        set_weights(c, 0.0);
        c->alpha = 0.5;   // no previous step: the first sampled interval is alpha_max (<= 1 = 2 * 0.5)
    }
    if (op & FIN_F0) {
        c->f[0] = f;
        c->resid = sqrt(f);
        if (!isfinite(f)) c->status |= DEV_NONFINITE;
    }
    if (op & FIN_N3CUR) c->n3max_cur = mx;
    if (op & FIN_AMAX) {
        c->n3max_next = mx;
        c->resid_prev = c->resid;
        const double m0 = c->n3max_cur, m1 = mx;
        double am = 1.0;
        if (m1 > m0) am = fmin(1.0, (n3_bound - m0) / (m1 - m0));
        c->alpha_max = am;
        c->alpha_fixed = alpha_fixed;
        if (alpha_fixed >= 0.0) {
            const double a = fmin(alpha_fixed, am);
            c->alpha = a;
            set_weights(c, a);
        } else {
            const double as = fmin(am, 2.0 * c->alpha);
            c->alpha_s = as;
            c->sample_alpha[0] = 0.5 * as;
            c->sample_alpha[1] = as;
            set_weights(c, 0.5 * as);
            set_weights(c + 1, 0.5 * as);
            set_weights(c + 2, as);
        }
    }
    if (op & FIN_F1) {
        c->f[1] = f;
        c->sample_alpha[1] = c->alpha_s;
        set_weights(c, c->alpha_s);
    }
    if (op & (FIN_F2_CHOOSE | FIN_F12_CHOOSE)) {
        // FIN_F12_CHOOSE: both samples' sums at once (f1 in red_sum, f2 in red_sum2); the z
        // passes of the samples recorded their status in the samples' blocks
        if (op & FIN_F12_CHOOSE) {
            c->f[1] = f;
            c->status |= c[1].status | c[2].status;
            c[1].status = 0;
            c[2].status = 0;
        }
        c->f[2] = (op & FIN_F12_CHOOSE) ? tot2 * inv_count : f;
        const double am = c->alpha_s, a = 0.5 * am;
        const double f0 = c->f[0], f1 = c->f[1], f2 = c->f[2];
        const double c2 = (f0 - 2.0 * f1 + f2) / (2.0 * a * a);
        const double c1 = (-3.0 * f0 + 4.0 * f1 - f2) / (2.0 * a);
        double al;
        if (c2 > 0.0) al = fmin(fmax(-c1 / (2.0 * c2), alpha_floor * am), am);
        else al = (f1 <= f2) ? a : am;
        c->alpha = al;
        set_weights(c, al);
    }
    if (op & FIN_ACCEPT) {
        c->f[3] = f;
        c->f[0] = f;
        c->resid = sqrt(f);
        c->n3max_cur = mx;
        c->iter += 1;
        if (!isfinite(f)) c->status |= DEV_NONFINITE;
    }
}

#endif  // DFT_DEFINE_FINALIZE

}  // namespace dftk
