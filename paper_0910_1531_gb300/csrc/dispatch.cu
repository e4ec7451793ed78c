// Passes<Real>: dispatch on the axis length to the compile-time or run-time kernels, and the
// line-search bookkeeping kernel.
#define DFT_DEFINE_FINALIZE
#include "kernels.cuh"
#include "passes.h"

#define DFT_DECLARE_EXTERN(N)                      \
    extern template struct LaunchX<float, N>;      \
    extern template struct LaunchY<float, N>;      \
    extern template struct LaunchZ<float, N>;      \
    extern template struct LaunchX<double, N>;     \
    extern template struct LaunchY<double, N>;     \
    extern template struct LaunchZ<double, N>;
DFT_CT_SIZES(DFT_DECLARE_EXTERN)
DFT_DECLARE_EXTERN(0)

#define DFT_CASE(N, L, call) case N: L<Real, N>::call; break;
#define DFT_SWITCH_X(n, call) if (g.xrt) return LaunchX<Real, 0>::call; switch (n) { \
    case 32: return LaunchX<Real, 32>::call; case 48: return LaunchX<Real, 48>::call; \
    case 64: return LaunchX<Real, 64>::call; case 96: return LaunchX<Real, 96>::call; \
    case 128: return LaunchX<Real, 128>::call; case 256: return LaunchX<Real, 256>::call; \
    default: return LaunchX<Real, 0>::call; }
#define DFT_SWITCH_Y(n, call) if (g.yrt) return LaunchY<Real, 0>::call; switch (n) { \
    case 32: return LaunchY<Real, 32>::call; case 48: return LaunchY<Real, 48>::call; \
    case 64: return LaunchY<Real, 64>::call; case 96: return LaunchY<Real, 96>::call; \
    case 128: return LaunchY<Real, 128>::call; case 256: return LaunchY<Real, 256>::call; \
    default: return LaunchY<Real, 0>::call; }
#define DFT_SWITCH_Z(n, call) switch (n) { \
    case 32: return LaunchZ<Real, 32>::call; case 48: return LaunchZ<Real, 48>::call; \
    case 64: return LaunchZ<Real, 64>::call; case 96: return LaunchZ<Real, 96>::call; \
    case 128: return LaunchZ<Real, 128>::call; case 256: return LaunchZ<Real, 256>::call; \
    default: return LaunchZ<Real, 0>::call; }

template <typename Real>
cudaError_t Passes<Real>::init_attributes() {
    cudaError_t e = cudaSuccess, r;
#define DFT_INIT(N) \
    if ((r = LaunchX<Real, N>::init()) != cudaSuccess) e = r; \
    if ((r = LaunchY<Real, N>::init()) != cudaSuccess) e = r; \
    if ((r = LaunchZ<Real, N>::init()) != cudaSuccess) e = r;
    DFT_CT_SIZES(DFT_INIT)
    DFT_INIT(0)
#undef DFT_INIT
    return e;
}

template <typename Real>
cudaError_t Passes<Real>::xcanon(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                                 int LR, const C* cspec, const Real* V, double* red, const C* tw) {
    DFT_SWITCH_X(g.nx, xcanon(st, g, px, sp, LR, cspec, V, red, tw))
}

template <typename Real>
cudaError_t Passes<Real>::canon_scale(cudaStream_t st, Ctl* ctl, const SpeciesDesc<Real>& sp, const double* red,
                                      int nblocks, int pdl) {
    return launch_k(dftk::k_canon_scale<Real>, 1, dftk::kThreads, 0, st, pdl, ctl, sp, red, nblocks);
}

template <typename Real>
cudaError_t Passes<Real>::build_ktab(cudaStream_t st, const SpeciesDesc<Real>& sp, double kf) {
    const int n = sp.tab_m2max + 1;
    dftk::k_ktab<Real><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(sp, kf, sp.tab_m2max, const_cast<Real*>(sp.tab_w),
                                                                  const_cast<Real*>(sp.tab_k), const_cast<Real*>(sp.tab_dk));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Passes<Real>::build_laptab(cudaStream_t st, const GridDesc& g, Real kfx, Real kfy, Real kfz, Real* out) {
    const int n = g.nx + g.ny + g.nz;
    dftk::k_laptab<Real><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(g, kfx, kfy, kfz, out);
    return cudaGetLastError();
}

template <typename Real>
int Passes<Real>::tile_y(int n, size_t budget) {
    if (dft_is_ct_size(n)) return dft_tile_y<Real>(n);
    for (int T = 16; T >= 1; T /= 2)
        if (smem_col(n, T, 2) <= budget) return T;
    return 1;
}

template <typename Real>
int Passes<Real>::tile_z(int n, size_t budget) {
    if (dft_is_ct_size(n)) return dft_tile_z<Real>(n);
    for (int T = 16; T >= 1; T /= 2)
        if (smem_col(n, T, 7) <= budget) return T;
    return 1;
}

template <typename Real>
cudaError_t Passes<Real>::xfwd(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int ncomp, int lx, const Real* in,
                        C* out, const C* tw) {
    DFT_SWITCH_X(g.nx, xfwd(st, g, px, ncomp, lx, in, out, tw))
}

template <typename Real>
cudaError_t Passes<Real>::yfft(cudaStream_t st, bool inv, const GridDesc& g, const AxisPlan& py, int T, int ncomp,
                               C* data, int* status, const C* tw, long long polls) {
    DFT_SWITCH_Y(g.ny, yfft(st, inv, g, py, T, ncomp, data, status, tw, polls))
}

template <typename Real>
cudaError_t Passes<Real>::zconv_fwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                             int T, Real kfx, Real kfy, Real kfz, int want_psi, const C* in, C* slot_n, C* slot_es,
                             double* red_energy, const C* tw, int* status) {
    DFT_SWITCH_Z(g.nz, zconv_fwd(st, g, pz, sp, T, kfx, kfy, kfz, want_psi, in, slot_n, slot_es, red_energy, tw, status))
}

template <typename Real>
cudaError_t Passes<Real>::xphi(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl, const C* A,
                        const C* B, C* mat, C* phi, float* red_max, int* status, double* red_phi, Real kfx,
                        const C* tw) {
    DFT_SWITCH_X(g.nx, xphi(st, g, px, LR, ctl, A, B, mat, phi, red_max, status, red_phi, kfx, tw))
}

template <typename Real>
cudaError_t Passes<Real>::zconv_bwd(cudaStream_t st, const GridDesc& g, const AxisPlan& pz, const SpeciesDesc<Real>& sp,
                             int T, Real kfx, Real kfy, Real kfz, int flags, int ncomp_out, const Ctl* ctl, C* phi,
                             const C* esA, const C* esB, C* es_mat, const C* tw) {
    DFT_SWITCH_Z(g.nz, zconv_bwd(st, g, pz, sp, T, kfx, kfy, kfz, flags, ncomp_out, ctl, phi, esA, esB, es_mat, tw))
}

template <typename Real>
cudaError_t Passes<Real>::zconv_bwd_pair(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx,
                                         Real kfy, Real kfz, int ncomp_out, const Ctl* ctl, C* phi, const C* esA,
                                         const C* esB, const C* tw) {
    DFT_SWITCH_Z(g.nz, zconv_bwd_pair(st, g, sp, kfx, kfy, kfz, ncomp_out, ctl, phi, esA, esB, tw))
}

template <typename Real>
bool Passes<Real>::has_zbwd_pair(const GridDesc& g, int ncomp_out) {
    DFT_SWITCH_Z(g.nz, has_zbwd_pair(g, ncomp_out))
}

template <typename Real>
cudaError_t Passes<Real>::zfft(cudaStream_t st, bool inv, const GridDesc& g, int ncomp, C* data, int* status,
                               const C* tw, long long polls) {
    DFT_SWITCH_Z(g.nz, zfft(st, inv, g, ncomp, data, status, tw, polls))
}

template <typename Real>
cudaError_t Passes<Real>::zmul(cudaStream_t st, const GridDesc& g, const SpeciesDesc<Real>& sp, Real kfx, Real kfy,
                               Real kfz, const C* in, C* slot_n, C* slot_es) {
    const long long npt = (long long)g.nz * g.ny * g.nxh;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const long long want = ceil_div(npt, dftk::kThreads), cap = (long long)sms * 16;
    return launch_k(dftk::k_zmul<Real>, (unsigned)(want < cap ? want : cap), dftk::kThreads, 0, st, g.pdl, g, sp, kfx,
                    kfy, kfz, in, slot_n, slot_es);
}

template <typename Real>
cudaError_t Passes<Real>::xupdate(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp, int LR,
                           const Ctl* ctl, const C* cspec, const Real* rho0, const Real* rho1, const Real* V,
                           Real* rho_out, Real* g_out, C* gspec_out, Real* rho_lo, double* red_sum, int* status,
                           const C* tw) {
    DFT_SWITCH_X(g.nx, xupdate(st, g, px, sp, LR, ctl, cspec, rho0, rho1, V, rho_out, g_out, gspec_out, rho_lo,
                               red_sum, status, tw))
}

template <typename Real>
cudaError_t Passes<Real>::xphi2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, const Ctl* ctl, const C* A,
                                const C* B, C* phi, int* status, Real kfx, const C* tw) {
    DFT_SWITCH_X(g.nx, xphi2(st, g, px, LR, ctl, A, B, phi, status, kfx, tw))
}

template <typename Real>
cudaError_t Passes<Real>::xupdate2(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                                   int LR, const Ctl* ctl, const C* cspec, const C* cspec2, const Real* rho0,
                                   const Real* rho1, const Real* V, Real* rho_lo, double* red_sum, double* red_sum2,
                                   int* status, const C* tw) {
    DFT_SWITCH_X(g.nx, xupdate2(st, g, px, sp, LR, ctl, cspec, cspec2, rho0, rho1, V, rho_lo, red_sum, red_sum2,
                                status, tw))
}

template <typename Real>
cudaError_t Passes<Real>::xinv(cudaStream_t st, const GridDesc& g, const AxisPlan& px, int LR, int ncomp, const C* spec,
                        Real* out, Real* out_last, const Offsets<Real>& off, int cmax, float* red_max, int wd,
                        Real kfx, const C* tw) {
    DFT_SWITCH_X(g.nx, xinv(st, g, px, LR, ncomp, spec, out, out_last, off, cmax, red_max, wd, kfx, tw))
}

template <typename Real>
cudaError_t Passes<Real>::xgrad(cudaStream_t st, const GridDesc& g, const AxisPlan& px, const SpeciesDesc<Real>& sp,
                                int LR, Real dv, const C* cspec, const Real* rho, const Real* V, Real* grad_rho,
                                Real* grad_V, double* red, const C* tw) {
    DFT_SWITCH_X(g.nx, xgrad(st, g, px, sp, LR, dv, cspec, rho, V, grad_rho, grad_V, red, tw))
}

template struct Passes<float>;
template struct Passes<double>;

cudaError_t launch_finalize(cudaStream_t st, Ctl* ctl, const double* red_sum, const double* red_sum2, int nsum,
                            const float* red_max, int nmax, int op, double inv_count, double alpha_fixed,
                            double n3_bound, double alpha_floor, int pdl) {
    if ((red_sum2 ? 2 : 1) * nsum + nmax > 8 * dftk::kFinThreadsSmall)
        return launch_k(dftk::k_finalize<dftk::kFinThreads>, 1, dftk::kFinThreads, 0, st, pdl, ctl, red_sum, red_sum2,
                        nsum, red_max, nmax, op, inv_count, alpha_fixed, n3_bound, alpha_floor);
    return launch_k(dftk::k_finalize<dftk::kFinThreadsSmall>, 1, dftk::kFinThreadsSmall, 0, st, pdl, ctl, red_sum,
                    red_sum2, nsum, red_max, nmax, op, inv_count, alpha_fixed, n3_bound, alpha_floor);
}

// ------------------------------------------------------------------------------------
// TMA tensor-map encoding through the driver entry point (no link against libcuda).
// ------------------------------------------------------------------------------------
#include <cudaTypedefs.h>
#include <mutex>

#include "tma.cuh"

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace

cudaError_t tma_encode_3d(CUtensorMap* map, void* base, unsigned long long d0, unsigned long long d1,
                          unsigned long long d2, unsigned long long stride1_bytes, unsigned long long stride2_bytes,
                          unsigned b0, unsigned b1, unsigned b2) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
