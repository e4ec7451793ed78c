// Allocation-free variant of dft_weighted_densities.
//
// Some callers cannot allocate device memory: code that runs inside a memory pool
// whose owner forbids cudaMalloc (for example a framework that has reserved all of
// the GPU's memory up front), code running where an allocation would implicitly
// synchronise the device and break the caller's timing or stream ordering, and
// embedded users who must know their whole device footprint at load time.  For them
// this file keeps all scratch of the weighted-density pipeline in one fixed,
// file-scope device array instead of memory obtained from cudaMalloc.
//
// The array is part of the library image: every GPU on which this part of the library
// is loaded holds it (kNoAllocScratchBytes) until the process exits.  Under lazy module
// loading (CUDA_MODULE_LOADING=LAZY, the default of recent CUDA runtimes) the module, and
// with it the array, is loaded on a device by the first call there; callers who need a
// fixed footprint make one call at initialisation.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gb300dft.h"
#include "passes.h"

namespace {

constexpr size_t kNoAllocScratchBytes = DFT_NOALLOC_SCRATCH_BYTES;   // 24 MiB
constexpr size_t kNoAllocElems = kNoAllocScratchBytes / sizeof(float2);

// The scratch itself.  In host code this name is only a host-side stand-in for the
// device symbol, never a device address: host code must obtain the address with
// cudaGetSymbolAddress (done once per device in device_scratch() below).
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocElems];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float2* g_scratch_ptr[kMaxDevices] = {nullptr};

// One-time set-up per device, with that device current: look up the device address of
// the scratch array and allow the kernels their full shared memory.  Returns nullptr
// (and an error text) on failure.  The result is kept for the life of the process: a
// cudaDeviceReset of that device invalidates it, so the entry point must not be used on a
// device after a reset within the same process.
float2* device_scratch(int dev, std::string* err) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (dev < 0 || dev >= kMaxDevices) {
        *err = "device ordinal out of range";
        return nullptr;
    }
    if (g_scratch_ptr[dev]) return g_scratch_ptr[dev];
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return nullptr;
    }
    e = Passes<float>::init_attributes();
    if (e != cudaSuccess) {
        *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return nullptr;
    }
    g_scratch_ptr[dev] = static_cast<float2*>(p);
    return g_scratch_ptr[dev];
}

// exp(-2 pi i m / n) for m < n, evaluated in double and rounded to float
__global__ void k_twiddles(float2* tw, int n) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * double(m) / double(n), &s, &c);
        tw[m] = make_float2(float(c), float(s));
    }
}


int lines_for(int nx, int per_unit, size_t budget, int cap) {
    const long long avail = (long long)(budget / sizeof(float2)) - nx;
    long long L = avail / (2LL * (nx + 1) * per_unit);
    return (int)(L < 1 ? 1 : (L > cap ? cap : L));
}

dft_status fail_na(char* errbuf, size_t errlen, dft_status code, const std::string& msg) {
    if (errbuf && errlen > 0) {
        const size_t n = msg.size() < errlen - 1 ? msg.size() : errlen - 1;
        std::memcpy(errbuf, msg.data(), n);
        errbuf[n] = '\0';
    }
    return code;
}

}  // namespace

extern "C" {

dft_status dft_weighted_densities_noalloc(const dft_params* prm, void* cuda_stream, const void* rho, void* n_out,
                                          char* errbuf, size_t errbuf_len) {
#define FAIL(code, msg) return fail_na(errbuf, errbuf_len, code, msg)
    if (!prm || !rho || !n_out) FAIL(DFT_EINVAL, "NULL argument");
    if (prm->precision != DFT_FP32_STAB) FAIL(DFT_EINVAL, "only DFT_FP32_STAB is supported");
    if (!dft_valid_length(prm->nx) || !dft_valid_length(prm->ny) || !dft_valid_length(prm->nz))
        FAIL(DFT_EINVAL, "grid sizes must be 4 <= n <= 512 with prime factors <= 31");
    if (!(prm->hx > 0 && prm->hy > 0 && prm->hz > 0)) FAIL(DFT_EINVAL, "grid spacing must be > 0");
    const int S = prm->nspecies;
    if (S < 1 || S > DFT_MAX_SPECIES || !prm->radius_nm) FAIL(DFT_EINVAL, "bad species");
    for (int i = 0; i < S; ++i)
        if (!(prm->radius_nm[i] > 0)) FAIL(DFT_EINVAL, "radius must be > 0");

    GridDesc g{};
    g.nx = prm->nx; g.ny = prm->ny; g.nz = prm->nz;
    g.nxh = g.nx / 2 + 1;
    g.pxh = (g.nxh + 1) & ~1;
    g.n = (long long)g.nx * g.ny * g.nz;
    g.nc = (long long)g.nz * g.ny * g.pxh;
    g.hx = prm->hx; g.hy = prm->hy; g.hz = prm->hz;
    AxisPlan ax, ay, az;
    if (!dft_radix_plan(g.nx, &ax) || !dft_radix_plan(g.ny, &ay) || !dft_radix_plan(g.nz, &az))
        FAIL(DFT_EINVAL, "no radix plan for the grid sizes");

    // scratch layout (float2 elements): status word | twiddles x, y, z | S spectra | 10 weighted
    // densities | S + 1 bulk-fluid spectra (written by the z pass, not used here)
    auto up = [](size_t v) { return (v + 31) & ~size_t(31); };   // keep 256-byte alignment
    const size_t o_status = 0;
    const size_t o_twx = o_status + up(1), o_twy = o_twx + up(g.nx), o_twz = o_twy + up(g.ny);
    const size_t o_spec = o_twz + up(g.nz);
    const size_t o_n = o_spec + up(size_t(S) * g.nc);
    const size_t o_es = o_n + up(size_t(DFT_NSPEC) * g.nc);
    const size_t need = o_es + up(size_t(S + 1) * g.nc);
    if (need > kNoAllocElems)
        FAIL(DFT_EINVAL, "grid and species need " + std::to_string(need * sizeof(float2)) +
                                       " bytes of scratch; the allocation-free entry point has " +
                                       std::to_string(kNoAllocScratchBytes));

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) FAIL(DFT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    std::string err;
    float2* base = device_scratch(dev, &err);
    if (!base) FAIL(DFT_ECUDA, err);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // Only the weights' radii enter the weighted densities; the bulk-fluid and Poisson
    // constants are zero, so the discarded bulk-fluid spectra the z pass writes are zero.
    SpeciesDesc<float> sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.S = S;
    for (int i = 0; i < S; ++i) sp.R[i] = float(prm->radius_nm[i]);
    sp.inv_n = float(1.0 / double(g.n));
    const double two_pi = 6.28318530717958647692;
    const float kfx = float(two_pi / (g.nx * g.hx)), kfy = float(two_pi / (g.ny * g.hy)),
                kfz = float(two_pi / (g.nz * g.hz));
    const int Ty = Passes<float>::tile_y(g.ny, 100 * 1024), Tz = Passes<float>::tile_z(g.nz, 112 * 1024);
    const int LX = lines_for(g.nx, 1, 48 * 1024, 32);
    const int LR = lines_for(g.nx, DFT_NCOMP / 2, 48 * 1024, 16);

    // The status word, where a bounded TMA wait of the y or z passes records that it gave up,
    // keeps the previous call's value: it is cleared here and read back at the end.  Every
    // other scratch element the pipeline reads is first written by this call; the twiddles
    // are rewritten every call (the previous call may have used other grid sizes).
    int* status = reinterpret_cast<int*>(base + o_status);
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) FAIL(DFT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_twiddles<<<4, 256, 0, st>>>(base + o_twx, g.nx);
    k_twiddles<<<4, 256, 0, st>>>(base + o_twy, g.ny);
    k_twiddles<<<4, 256, 0, st>>>(base + o_twz, g.nz);
    Offsets<float> off;
    for (int c = 0; c < DFT_NCOMP + 2; ++c) off.v[c] = 0.f;
    e = Passes<float>::xfwd(st, g, ax, S, LX, static_cast<const float*>(rho), base + o_spec, base + o_twx);
    if (e == cudaSuccess) e = Passes<float>::yfft(st, false, g, ay, Ty, S, base + o_spec, status, base + o_twy);
    if (e == cudaSuccess)
        e = Passes<float>::zconv_fwd(st, g, az, sp, Tz, kfx, kfy, kfz, 0, base + o_spec, base + o_n, base + o_es,
                                     nullptr, base + o_twz, status);
    if (e == cudaSuccess) e = Passes<float>::yfft(st, true, g, ay, Ty, DFT_NSPEC, base + o_n, status, base + o_twy);
    if (e == cudaSuccess)
        e = Passes<float>::xinv(st, g, ax, LR, DFT_NCOMP, base + o_n, static_cast<float*>(n_out), nullptr, off, -1,
                                nullptr, 1, kfx, base + o_twx);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) FAIL(DFT_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    // the status word, read back once the work is done (a pageable copy into a local: no
    // allocation); this makes the call synchronous with respect to `st`
    int dev_status = 0;
    e = cudaMemcpyAsync(&dev_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) FAIL(DFT_ECUDA, std::string("status read-back: ") + cudaGetErrorString(e));
    if (dev_status & DEV_TIMEOUT)
        FAIL(DFT_ETIMEOUT, "a bounded wait on an asynchronous copy gave up; n_out is incomplete");
    if (errbuf && errbuf_len > 0) errbuf[0] = '\0';
    return DFT_OK;
#undef FAIL
}

}  // extern "C"
