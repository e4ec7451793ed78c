// C ABI of the GB300 classical-DFT library: plan creation, the FFT/Picard entry points
// and per-kernel profiling.  All device work is queued on the plan's stream; the
// Picard iteration keeps its scalars (mixing weights, residuals, alpha) in a device
// control block so an iteration needs no host round trip.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bulk.h"
#include "fft.cuh"
#include "gb300dft.h"
#include "newton.h"
#include "passes.h"

namespace {

enum Kind { K_XFWD, K_YFFT, K_ZFWD, K_XPHI, K_ZBWD, K_XUPD, K_XINV, K_FIN, K_ZFFT, K_ZMUL, K_COUNT };
const char* kKindNames[K_COUNT] = {"xfwd", "yfft", "zconv_fwd", "xphi", "zconv_bwd", "xupdate", "xinv", "finalize",
                                   "zfft", "zmul"};

constexpr double kN3Bound = 0.9;       // Sec. "Nonlinear solver"
constexpr double kAlphaFloor = 1e-3;   // lower clamp of the parabola minimiser, in units of alpha_max

std::string g_create_error;

struct ProfRec {
    int kind;
    double bytes;
    cudaEvent_t a, b;
};

}  // namespace

struct dft_plan {
    int S = 0;
    int precision = DFT_FP32_STAB;
    std::vector<double> R, z, molar;
    std::vector<double> n_fixed;    // particles of fixed-number species (0: bath species)
    int ncanon = 0;
    double* red_canon = nullptr;    // [blocks][DFT_MAXS] normalisation partial sums
    double T = 0, eps_r = 0;
    BathState bath;
    GridDesc g{};
    AxisPlan ax{}, ay{}, az{};
    double kf[3] = {0, 0, 0};
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t csize = 0, rsize = 0;
    void* tw[3] = {nullptr, nullptr, nullptr};
    void* T1 = nullptr;
    void* slotA = nullptr;
    void* slotB = nullptr;
    void* gbuf = nullptr;
    // x half spectra of gbuf's G, written by the update pass that forms G in dft_iter_begin /
    // dft_iter_step (nothing else writes it): the next iteration's first half starts from them
    void* gspec = nullptr;
    void* rho_lo = nullptr;         // FP32 plans: low part of the extended iterate of dft_iter_*
    void* stage_rho = nullptr;
    void* stage_V = nullptr;
    double* red_sum = nullptr;
    double* red_sum2 = nullptr;     // the second line-search sample's partial sums (paired samples)
    float* red_max = nullptr;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;
    int Ty = 1, Tz = 1, LX = 1, LRphi = 1, LRupd = 1;
    int LRphi2 = 1, LRupd2 = 1;     // rows per block of the paired-sample x passes
    int LRn3 = 0;                   // rows per block of the n3-maximum x pass (0: from the budget)
    SpeciesDesc<float> spf{};
    SpeciesDesc<double> spd{};
    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> evpool;
    size_t ev_used = 0;
    int prof_launches[K_COUNT] = {0};
    double prof_ms[K_COUNT] = {0};
    double prof_bytes[K_COUNT] = {0};
    std::string err;
    void* ktab = nullptr;           // |k| tables of the compile-time z passes (cubic boxes)
    void* laptab = nullptr;         // per-axis Laplacian terms of the Poisson kernel (SpeciesDesc::lap1d)
    cudaStream_t cap = nullptr;     // capture stream of the one-iteration graph (dft_iter_run)
    cudaStream_t side = nullptr;    // copy stream of dft_picard_step_host
    cudaEvent_t v_ready = nullptr;  // V staged (dft_picard_step_host)
    cudaGraph_t igraph = nullptr;
    cudaGraphExec_t iexec = nullptr;
    const void* graph_rho = nullptr;
    const void* graph_V = nullptr;
    double graph_alpha = 0.0;
    bool iloop = false;             // the cached graph is the on-device loop (else one iteration)
    std::string tuning;             // the transform variants and rows per block in use (text)
    double* grad_red = nullptr;     // partial sums of dft_grad (allocated on first use)
    size_t grad_red_len = 0;
    bool iter_ready = false;
    const void* iter_rho = nullptr;
    const void* iter_V = nullptr;
    long long wait_polls = DFT_WAIT_POLLS;   // bound of the y passes' TMA tile waits
    bool pdl_on = true;             // programmatic dependent launch of the passes (off while profiling)

    long long blocks_x(int LR) const { return ceil_div((long long)g.ny * g.nz, LR); }
};

namespace {

dft_status fail(dft_plan* p, dft_status code, const std::string& msg) {
    if (p) p->err = msg;
    else g_create_error = msg;
    return code;
}


// Shared-memory budget of a pass's row block (bytes); a positive environment value overrides it.
size_t env_budget(const char* name, size_t dflt) {
    const char* v = std::getenv(name);
    if (!v) return dflt;
    const long long x = std::atoll(v);
    return x > 0 ? size_t(x) : dflt;
}

int pick_lines(int nx, size_t csize, int lines_per_unit, size_t budget, int cap) {
    const long long avail = (long long)(budget / csize) - nx;
    long long L = avail / (2LL * (nx + 1) * lines_per_unit);
    if (L < 1) L = 1;
    if (L > cap) L = cap;
    return (int)L;
}

template <typename Real> SpeciesDesc<Real>& species(dft_plan* p);
template <> SpeciesDesc<float>& species<float>(dft_plan* p) { return p->spf; }
template <> SpeciesDesc<double>& species<double>(dft_plan* p) { return p->spd; }

template <typename Real> void fill_species(dft_plan* p) {
    SpeciesDesc<Real>& sp = species<Real>(p);
    memset(&sp, 0, sizeof(sp));
    const BathState& b = p->bath;
    const double pi = 3.14159265358979323846;
    sp.S = p->S;
    for (int i = 0; i < p->S; ++i) {
        sp.R[i] = Real(p->R[i]);
        sp.z[i] = Real(p->z[i]);
        sp.rho_b[i] = Real(b.rho[i]);
        sp.inv_rho_b[i] = b.rho[i] > 0 ? Real(1.0 / b.rho[i]) : Real(0);
        sp.mu_hs_b[i] = Real(b.mu_hs[i]);
        sp.mu_ex_b[i] = Real(b.mu_hs[i] + b.mu_es[i]);
        sp.n_rho_b[i] = Real(double(p->g.n) * b.rho[i]);
        if (p->n_fixed[i] > 0.0) {
            const double dv = p->g.hx * p->g.hy * p->g.hz;
            sp.canon[i] = 1;
            sp.nfix_dv[i] = p->n_fixed[i] / dv;
            sp.inv_rho_b[i] = Real(double(p->g.n) * dv / p->n_fixed[i]);   // 1 / mean density
            sp.ncanon += 1;
        }
    }
    for (int i = 0; i < p->S; ++i)
        for (int j = 0; j < p->S; ++j) {
            const double li = b.lam[i], lj = b.lam[j];
            sp.es_pref[i][j] = Real(0.5 * b.lb * p->z[i] * p->z[j]);
            if (b.gamma > 0.0) {
                sp.es_a[i][j] = Real(1.0 / (2.0 * li * lj));
                sp.es_b[i][j] = Real((li + lj) / (li * lj));
                sp.es_c[i][j] = Real((li - lj) * (li - lj) / (2.0 * li * lj) + 2.0);
            } else {   // Gamma = 0: l -> infinity leaves the Coulomb term 2/r
                sp.es_a[i][j] = Real(0);
                sp.es_b[i][j] = Real(0);
                sp.es_c[i][j] = Real(2);
            }
            sp.es_R[i][j] = Real(p->R[i] + p->R[j]);
            if (b.gamma > 0.0) {
                // l = R + s, s = 1/(2 Gamma): d/dGamma = d/ds * (-1 / (2 Gamma^2))
                const double dsdg = -0.5 / (b.gamma * b.gamma);
                const double li2lj2 = li * li * lj * lj;
                const double dR = p->R[i] - p->R[j];
                sp.es_da[i][j] = Real(-(li + lj) / (2.0 * li2lj2) * dsdg);
                sp.es_db[i][j] = Real(-(1.0 / (li * li) + 1.0 / (lj * lj)) * dsdg);
                sp.es_dc[i][j] = Real(-dR * dR * (li + lj) / (2.0 * li2lj2) * dsdg);
            } else {
                sp.es_da[i][j] = sp.es_db[i][j] = sp.es_dc[i][j] = Real(0);
            }
            sp.pois[i][j] = Real(4.0 * pi * b.lb * p->z[i] * p->z[j]);
        }
    sp.inv_n = Real(1.0 / double(p->g.n));
    sp.coulomb_limit = b.gamma > 0.0 ? 0 : 1;
}

template <typename C> void fill_twiddles(int n, std::vector<C>* out) {
    out->resize(n);
    const double two_pi = 6.28318530717958647692;
    for (int m = 0; m < n; ++m) {
        const double a = -two_pi * double(m) / double(n);
        (*out)[m].x = decltype(C().x)(std::cos(a));
        (*out)[m].y = decltype(C().x)(std::sin(a));
    }
}

// --------------------------------------------------------------------------------------
// profiling helpers
// --------------------------------------------------------------------------------------
// profiled launches whose event pairs are kept before their times are collected
constexpr size_t kProfBatch = 4096;

cudaEvent_t take_event(dft_plan* p) {
    if (p->ev_used == p->evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        p->evpool.push_back(e);
    }
    return p->evpool[p->ev_used++];
}

struct Prof {
    dft_plan* p;
    int kind;
    double bytes;
    cudaEvent_t a = nullptr;
    Prof(dft_plan* pp, int k, double by) : p(pp), kind(k), bytes(by) {
        if (p->prof) {
            a = take_event(p);
            cudaEventRecord(a, p->stream);
        }
    }
    ~Prof() {
        if (p->prof) {
            cudaEvent_t b = take_event(p);
            cudaEventRecord(b, p->stream);
            p->recs.push_back({kind, bytes, a, b});
        }
    }
};

// bytes of one complex half-spectrum component (used elements, not the row padding) and of
// one real field component
double CB(const dft_plan* p) { return double(p->g.nz) * p->g.ny * p->g.nxh * double(p->csize); }
double RB(const dft_plan* p) { return double(p->g.n) * double(p->rsize); }

void collect_profile(dft_plan* p) {
    if (p->recs.empty()) return;
    cudaStreamSynchronize(p->stream);
    for (const ProfRec& r : p->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p->prof_launches[r.kind] += 1;
            p->prof_ms[r.kind] += ms;
            p->prof_bytes[r.kind] += r.bytes;
        }
    }
    p->recs.clear();
    p->ev_used = 0;
}

// Queue one kernel; `bytes` is its algorithmic global traffic (each input element read once,
// each output element written once), accumulated by the profiler.
#define LAUNCH(p, kind, bytes, call)                                                          \
    do {                                                                                      \
        cudaError_t _e;                                                                       \
        {                                                                                     \
            Prof _pr((p), (kind), double(bytes));                                             \
            _e = (call);                                                                      \
        }                                                                                     \
        if (_e == cudaSuccess) _e = cudaGetLastError();                                       \
        if (_e != cudaSuccess)                                                                \
            return fail((p), DFT_ECUDA, std::string(kKindNames[kind]) + ": " + cudaGetErrorString(_e)); \
        if ((p)->prof && (p)->recs.size() > kProfBatch) collect_profile(p);                   \
    } while (0)

// --------------------------------------------------------------------------------------
// sequences
// --------------------------------------------------------------------------------------
template <typename Real> struct Ops {
    using C = typename Cplx<Real>::type;
    using P = Passes<Real>;

    static const C* tw(dft_plan* p, int a) { return static_cast<const C*>(p->tw[a]); }
    static C* T1(dft_plan* p) { return static_cast<C*>(p->T1); }
    static C* slot_n(void* s) { return static_cast<C*>(s); }
    static C* slot_es(dft_plan* p, void* s) { return static_cast<C*>(s) + DFT_NSPEC * p->g.nc; }
    static Real kf(dft_plan* p, int a) { return Real(p->kf[a]); }

    // rho (S real fields) -> slot: ten weighted densities (kx, ky, z) and the S (+psi)
    // bulk-fluid / Poisson spectra (kx, ky, kz)
    // pre (or nullptr): rho's x half spectra, already formed (the update pass that computed rho
    // as G wrote them); the y and z passes then transform them in place
    static dft_status first_half(dft_plan* p, const Real* rho, void* slot, int want_psi,
                                 double* red_energy = nullptr, C* pre = nullptr) {
        const SpeciesDesc<Real>& sp = species<Real>(p);
        C* W = pre ? pre : T1(p);
        if (!pre)
            LAUNCH(p, K_XFWD, p->S * (RB(p) + CB(p)), P::xfwd(p->stream, p->g, p->ax, p->S, p->LX, rho, W, tw(p, 0)));
        LAUNCH(p, K_YFFT, 2.0 * (p->S) * CB(p), P::yfft(p->stream, false, p->g, p->ay, p->Ty, p->S, W, &p->ctl->status, tw(p, 1), p->wait_polls));
        if (p->g.zsplit && dft_is_ct_size(p->g.nz) && !want_psi && !red_energy) {
            // z forward transform of the species, the k-space products, z inverse of the nine
            LAUNCH(p, K_ZFFT, 2.0 * p->S * CB(p),
                   P::zfft(p->stream, false, p->g, p->S, W, &p->ctl->status, tw(p, 2), p->wait_polls));
            LAUNCH(p, K_ZMUL, (p->S + DFT_NSPEC + p->S) * CB(p),
                   P::zmul(p->stream, p->g, sp, kf(p, 0), kf(p, 1), kf(p, 2), W, slot_n(slot), slot_es(p, slot)));
            LAUNCH(p, K_ZFFT, 2.0 * DFT_NSPEC * CB(p),
                   P::zfft(p->stream, true, p->g, DFT_NSPEC, slot_n(slot), &p->ctl->status, tw(p, 2), p->wait_polls));
        } else {
            LAUNCH(p, K_ZFWD, (p->S + DFT_NSPEC + p->S + want_psi) * CB(p),
                   P::zconv_fwd(p->stream, p->g, p->az, sp, p->Tz, kf(p, 0), kf(p, 1), kf(p, 2), want_psi, W,
                                slot_n(slot), slot_es(p, slot), red_energy, tw(p, 2), &p->ctl->status));
        }
        LAUNCH(p, K_YFFT, 2.0 * (DFT_NSPEC) * CB(p), P::yfft(p->stream, true, p->g, p->ay, p->Ty, DFT_NSPEC, slot_n(slot), &p->ctl->status, tw(p, 1), p->wait_polls));
        return DFT_OK;
    }

    // weighted densities mixed from slot A (and slot B) -> G at rho = w0 rho0 + w1 rho1
    // rho_lo (FP32 iterations, else nullptr): low part of the extended iterate rho0 + rho_lo
    // gspec_out (or nullptr): G's x half spectra too (the next first half's input)
    static dft_status second_half(dft_plan* p, bool use_B, bool materialise, const Real* rho0, const Real* rho1,
                                  const Real* V, Real* rho_out, Real* g_out, Real* rho_lo = nullptr,
                                  C* gspec_out = nullptr) {
        const SpeciesDesc<Real>& sp = species<Real>(p);
        C* A = slot_n(p->slotA);
        C* B = use_B ? slot_n(p->slotB) : nullptr;
        C* esA = slot_es(p, p->slotA);
        C* esB = use_B ? slot_es(p, p->slotB) : nullptr;
        LAUNCH(p, K_XPHI, ((use_B ? 2 : 1) + 1 + (materialise ? 1 : 0)) * DFT_NSPEC * CB(p),
               P::xphi(p->stream, p->g, p->ax, p->LRphi, p->ctl, A, B, materialise ? A : nullptr, T1(p),
                                  p->red_max, &p->ctl->status, nullptr, kf(p, 0), tw(p, 0)));
        LAUNCH(p, K_YFFT, 2.0 * (DFT_NSPEC) * CB(p), P::yfft(p->stream, false, p->g, p->ay, p->Ty, DFT_NSPEC, T1(p), &p->ctl->status, tw(p, 1), p->wait_polls));
        LAUNCH(p, K_ZBWD, (DFT_NSPEC + p->S * ((use_B ? 2 : 1) + 1 + (materialise ? 1 : 0))) * CB(p),
               P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, kf(p, 0), kf(p, 1), kf(p, 2), 3, p->S,
                                       p->ctl, T1(p), esA, esB, materialise ? esA : nullptr, tw(p, 2)));
        LAUNCH(p, K_YFFT, 2.0 * (p->S) * CB(p), P::yfft(p->stream, true, p->g, p->ay, p->Ty, p->S, T1(p), &p->ctl->status, tw(p, 1), p->wait_polls));
        if (p->ncanon > 0) {
            // fixed-number species: the sum of their Boltzmann factors first (its reciprocal
            // scales G in the update pass)
            LAUNCH(p, K_XUPD, p->ncanon * (CB(p) + RB(p)),
                   P::xcanon(p->stream, p->g, p->ax, sp, p->LRupd, T1(p), V, p->red_canon, tw(p, 0)));
            LAUNCH(p, K_FIN, p->blocks_x(p->LRupd) * DFT_MAXS * 8.0,
                   P::canon_scale(p->stream, p->ctl, sp, p->red_canon, (int)p->blocks_x(p->LRupd), p->g.pdl));
        }
        LAUNCH(p, K_XUPD, p->S * (CB(p) * (gspec_out ? 2 : 1) +
                                  RB(p) * ((rho1 ? 2 : 1) + 1 + (rho_out ? 1 : 0) + (g_out ? 1 : 0) +
                                           (rho_lo ? (rho_out ? 2 : 1) : 0))),
               P::xupdate(p->stream, p->g, p->ax, sp, p->LRupd, p->ctl, T1(p), rho0, rho1, V, rho_out,
                          g_out, gspec_out, rho_lo, p->red_sum, &p->ctl->status, tw(p, 0)));
        return DFT_OK;
    }

    // The two line-search samples rho0 + a_m (rho1 - rho0), a_1 = alpha_s / 2, a_2 = alpha_s (weights
    // in ctl[1], ctl[2], set by FIN_AMAX), evaluated together: one Phi' x pass for both mixtures of
    // the slots (one read of slots A and B), one y pass over the 18 Phi' spectra, one z pass for
    // both (the persistent TMA pass; else one per sample), one y pass over the 2 S correlation
    // spectra (else one per sample), and one update pass reading rho0, rho1, V (and the low part)
    // once for both residual sums (red_sum, red_sum2).  Nothing is written to rho or G.
    static dft_status second_half_pair(dft_plan* p, const Real* rho0, const Real* rho1, const Real* V, Real* rho_lo) {
        const SpeciesDesc<Real>& sp = species<Real>(p);
        C* A = slot_n(p->slotA);
        C* B = slot_n(p->slotB);
        C* esA = slot_es(p, p->slotA);
        C* esB = slot_es(p, p->slotB);
        C* T2 = T1(p) + (long long)DFT_NSPEC * p->g.nc;   // the second sample's spectra
        LAUNCH(p, K_XPHI, 4.0 * DFT_NSPEC * CB(p),
               P::xphi2(p->stream, p->g, p->ax, p->LRphi2, p->ctl, A, B, T1(p), &p->ctl->status, kf(p, 0), tw(p, 0)));
        LAUNCH(p, K_YFFT, 2.0 * (2 * DFT_NSPEC) * CB(p),
               P::yfft(p->stream, false, p->g, p->ay, p->Ty, 2 * DFT_NSPEC, T1(p), &p->ctl->status, tw(p, 1),
                       p->wait_polls));
        C* c2 = T2;   // the second sample's correlation spectra
        if (P::has_zbwd_pair(p->g, p->S)) {
            // one z pass for both samples (the ES tiles read once; sample 2's results after sample
            // 1's, at T1 components S .. 2 S - 1), then one y inverse over the 2 S components
            LAUNCH(p, K_ZBWD, (2.0 * DFT_NSPEC + 4.0 * p->S) * CB(p),
                   P::zconv_bwd_pair(p->stream, p->g, sp, kf(p, 0), kf(p, 1), kf(p, 2), p->S, p->ctl + 1, T1(p), esA,
                                     esB, tw(p, 2)));
            LAUNCH(p, K_YFFT, 2.0 * (2 * p->S) * CB(p),
                   P::yfft(p->stream, true, p->g, p->ay, p->Ty, 2 * p->S, T1(p), &p->ctl->status, tw(p, 1),
                           p->wait_polls));
            c2 = T1(p) + (long long)p->S * p->g.nc;
        } else {
            for (int m = 0; m < 2; ++m) {
                C* phi = m == 0 ? T1(p) : T2;
                LAUNCH(p, K_ZBWD, (DFT_NSPEC + p->S * 3) * CB(p),
                       P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, kf(p, 0), kf(p, 1), kf(p, 2), 3, p->S,
                                    p->ctl + 1 + m, phi, esA, esB, nullptr, tw(p, 2)));
                LAUNCH(p, K_YFFT, 2.0 * (p->S) * CB(p),
                       P::yfft(p->stream, true, p->g, p->ay, p->Ty, p->S, phi, &p->ctl->status, tw(p, 1),
                               p->wait_polls));
            }
        }
        LAUNCH(p, K_XUPD, 2.0 * p->S * CB(p) + p->S * RB(p) * (3 + (rho_lo ? 1 : 0)),
               P::xupdate2(p->stream, p->g, p->ax, sp, p->LRupd2, p->ctl, T1(p), c2, rho0, rho1, V, rho_lo,
                           p->red_sum, p->red_sum2, &p->ctl->status, tw(p, 0)));
        return DFT_OK;
    }

    static dft_status xinv(dft_plan* p, int ncomp, const C* spec, Real* out, Real* out_last, const double* offs,
                           int cmax, float* red_max, int* blocks_out) {
        const int lpr = (ncomp + 1) / 2;
        const int LR = (ncomp == 1 && p->LRn3 > 0) ? p->LRn3 : pick_lines(p->g.nx, sizeof(C), lpr, 48 * 1024, 16);
        Offsets<Real> off;
        for (int c = 0; c < DFT_NCOMP + 2; ++c) off.v[c] = Real(0);
        if (offs)
            for (int c = 0; c < ncomp; ++c) off.v[c] = Real(offs[c]);
        // ten real rows are the weighted densities, built from the nine kept spectra
        const int wd = ncomp == DFT_NCOMP ? 1 : 0;
        LAUNCH(p, K_XINV, ((wd ? DFT_NSPEC : ncomp) * CB(p) + (out || out_last ? ncomp * RB(p) : 0.0)),
               P::xinv(p->stream, p->g, p->ax, LR, ncomp, spec, out, out_last, off, cmax, red_max, wd, kf(p, 0),
                       tw(p, 0)));
        if (blocks_out) *blocks_out = (int)p->blocks_x(LR);
        return DFT_OK;
    }
};

dft_status finalize(dft_plan* p, int op, int nsum, int nmax, double alpha_fixed, bool pair = false) {
    const double inv_count = 1.0 / (double(p->S) * double(p->g.n));
    LAUNCH(p, K_FIN, (pair ? 2 : 1) * nsum * 8.0 + nmax * 4.0,
           launch_finalize(p->stream, p->ctl, p->red_sum, pair ? p->red_sum2 : nullptr, nsum, p->red_max, nmax, op,
                           inv_count, alpha_fixed, kN3Bound, kAlphaFloor, p->g.pdl));
    return DFT_OK;
}

dft_status read_ctl(dft_plan* p) {
    cudaError_t e = cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("reading control block: ") + cudaGetErrorString(e));
    // a timeout first: the passes after it ran on unfinished spectra
    if (p->ctl_host->status & DEV_TIMEOUT) return fail(p, DFT_ETIMEOUT, "a bounded wait on an asynchronous copy gave up");
    if (p->ctl_host->status & DEV_N3BOUND) return fail(p, DFT_EN3BOUND, "local packing fraction n3 >= 1 met");
    if (p->ctl_host->status & DEV_NONFINITE) return fail(p, DFT_ENONFINITE, "non-finite density or residual met");
    return DFT_OK;
}

dft_status reset_status(dft_plan* p) {
    // the iteration's status word and those of the two samples' blocks
    cudaError_t e = cudaSuccess;
    for (int m = 0; m < 3 && e == cudaSuccess; ++m) e = cudaMemsetAsync(&p->ctl[m].status, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
    return DFT_OK;
}

#define TRY(x)                        \
    do {                              \
        dft_status _s = (x);          \
        if (_s != DFT_OK) return _s;  \
    } while (0)

// v_ready (optional): an event the second half (the first use of V) waits for
template <typename Real> dft_status iter_begin_t(dft_plan* p, Real* rho, const Real* V, cudaEvent_t v_ready = nullptr) {
    using O = Ops<Real>;
    using C = typename Cplx<Real>::type;
    TRY(reset_status(p));
    // the extended iterate starts as the caller's rho with a zero low part
    if (p->rho_lo && cudaMemsetAsync(p->rho_lo, 0, size_t(p->S) * p->g.n * sizeof(Real), p->stream) != cudaSuccess)
        return fail(p, DFT_ECUDA, "memset of the iterate's low part");
    TRY(O::first_half(p, rho, p->slotA, 0));
    TRY(finalize(p, FIN_IDENTITY, 0, 0, -1.0));
    if (v_ready && cudaStreamWaitEvent(p->stream, v_ready, 0) != cudaSuccess)
        return fail(p, DFT_ECUDA, "stream wait");
    TRY(O::second_half(p, false, false, rho, nullptr, V, nullptr, static_cast<Real*>(p->gbuf), nullptr,
                       static_cast<C*>(p->gspec)));
    TRY(finalize(p, FIN_F0 | FIN_N3CUR, (int)p->blocks_x(p->LRupd), (int)p->blocks_x(p->LRphi), -1.0));
    p->iter_ready = true;
    p->iter_rho = rho;
    p->iter_V = V;
    return DFT_OK;
}

template <typename Real> dft_status iter_step_t(dft_plan* p, Real* rho, const Real* V, double alpha) {
    using O = Ops<Real>;
    using C = typename Cplx<Real>::type;
    Real* g = static_cast<Real*>(p->gbuf);
    C* gspec = static_cast<C*>(p->gspec);
    // the first half of G's weighted densities starts from G's x spectra (written by the update
    // pass that formed G: the previous step's accepted point, or dft_iter_begin)
    TRY(O::first_half(p, g, p->slotB, 0, nullptr, gspec));
    int nb = 0;
    TRY(O::xinv(p, 1, O::slot_n(p->slotB) + 3 * p->g.nc, nullptr, nullptr, nullptr, 0, p->red_max, &nb));
    TRY(finalize(p, FIN_AMAX, 0, nb, alpha));
    const int nsum = (int)p->blocks_x(p->LRupd);
    Real* lo = static_cast<Real*>(p->rho_lo);
    if (alpha < 0.0 && p->ncanon == 0) {
        // both samples in one paired evaluation (their points are known before either is
        // evaluated); fixed-number species need the normalisation of each sample first, so
        // those plans take the samples one after the other
        TRY(O::second_half_pair(p, rho, g, V, lo));
        TRY(finalize(p, FIN_F12_CHOOSE, (int)p->blocks_x(p->LRupd2), 0, alpha, true));
    } else if (alpha < 0.0) {
        TRY(O::second_half(p, true, false, rho, g, V, nullptr, nullptr, lo));
        TRY(finalize(p, FIN_F1, nsum, 0, alpha));
        TRY(O::second_half(p, true, false, rho, g, V, nullptr, nullptr, lo));
        TRY(finalize(p, FIN_F2_CHOOSE, nsum, 0, alpha));
    }
    TRY(O::second_half(p, true, true, rho, g, V, rho, g, lo, gspec));
    TRY(finalize(p, FIN_ACCEPT, nsum, (int)p->blocks_x(p->LRphi), alpha));
    (void)sizeof(C);
    return DFT_OK;
}

dft_status check_plan(dft_plan* p) {
    if (!p) return fail(nullptr, DFT_EINVAL, "NULL plan");
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur == p->device) return DFT_OK;
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return DFT_OK;
}

bool is_fp64(const dft_plan* p) { return p->precision == DFT_FP64; }

template <typename Real> dft_status c1_hs_t(dft_plan* p, const Real* rho, Real* c1) {
    using O = Ops<Real>;
    using P = Passes<Real>;
    const SpeciesDesc<Real>& sp = species<Real>(p);
    TRY(O::first_half(p, rho, p->slotA, 0));
    TRY(finalize(p, FIN_IDENTITY, 0, 0, -1.0));
    LAUNCH(p, K_XPHI, 2.0 * DFT_NSPEC * CB(p), P::xphi(p->stream, p->g, p->ax, p->LRphi, p->ctl, O::slot_n(p->slotA), nullptr, nullptr,
                              O::T1(p), p->red_max, &p->ctl->status, nullptr, O::kf(p, 0), O::tw(p, 0)));
    LAUNCH(p, K_YFFT, 2.0 * (DFT_NSPEC) * CB(p), P::yfft(p->stream, false, p->g, p->ay, p->Ty, DFT_NSPEC, O::T1(p), &p->ctl->status, O::tw(p, 1), p->wait_polls));
    LAUNCH(p, K_ZBWD, (DFT_NSPEC + p->S) * CB(p), P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 1, p->S,
                                   p->ctl, O::T1(p), O::slot_es(p, p->slotA), nullptr, nullptr, O::tw(p, 2)));
    LAUNCH(p, K_YFFT, 2.0 * (p->S) * CB(p), P::yfft(p->stream, true, p->g, p->ay, p->Ty, p->S, O::T1(p), &p->ctl->status, O::tw(p, 1), p->wait_polls));
    TRY(O::xinv(p, p->S, O::T1(p), c1, nullptr, nullptr, -1, nullptr, nullptr));
    return DFT_OK;
}

template <typename Real> dft_status c1_es_t(dft_plan* p, const Real* rho, Real* c1, Real* psi) {
    using O = Ops<Real>;
    using P = Passes<Real>;
    const SpeciesDesc<Real>& sp = species<Real>(p);
    const int want_psi = psi ? 1 : 0;
    const int nout = p->S + want_psi;
    TRY(O::first_half(p, rho, p->slotA, want_psi));
    TRY(finalize(p, FIN_IDENTITY, 0, 0, -1.0));
    LAUNCH(p, K_ZBWD, 2.0 * nout * CB(p), P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 2, nout,
                                   p->ctl, O::T1(p), O::slot_es(p, p->slotA), nullptr, nullptr, O::tw(p, 2)));
    LAUNCH(p, K_YFFT, 2.0 * (nout) * CB(p), P::yfft(p->stream, true, p->g, p->ay, p->Ty, nout, O::T1(p), &p->ctl->status, O::tw(p, 1), p->wait_polls));
    double offs[DFT_NCOMP + 2] = {0};
    for (int s = 0; s < p->S; ++s) offs[s] = -p->bath.mu_es[s];
    TRY(O::xinv(p, nout, O::T1(p), c1, psi, offs, -1, nullptr, nullptr));
    return DFT_OK;
}

template <typename Real> dft_status picard_map_t(dft_plan* p, const Real* rho, const Real* V, Real* g) {
    using O = Ops<Real>;
    TRY(reset_status(p));
    TRY(O::first_half(p, rho, p->slotA, 0));
    TRY(finalize(p, FIN_IDENTITY, 0, 0, -1.0));
    TRY(O::second_half(p, false, false, rho, nullptr, V, nullptr, g));
    TRY(finalize(p, FIN_F0 | FIN_N3CUR, (int)p->blocks_x(p->LRupd), (int)p->blocks_x(p->LRphi), -1.0));
    return DFT_OK;
}

// Bath derivatives by central differences of the host bath solver, Richardson-extrapolated
// (h and h/2), in units of the number density: d/drho_bath_k = d/dc_k / 0.602214076.
struct BathDerivs {
    std::vector<double> dmu_ex;   // [i * S + k] = d beta mu_ex_bath_i / d rho_bath_k
    std::vector<double> dmu_es;   // [i * S + k]
    std::vector<double> dgamma;   // [k]
};

bool bath_derivatives(dft_plan* p, BathDerivs* d, std::string* err) {
    const int S = p->S;
    d->dmu_ex.assign(S * S, 0.0);
    d->dmu_es.assign(S * S, 0.0);
    d->dgamma.assign(S, 0.0);
    const double to_rho = 0.602214076;
    for (int k = 0; k < S; ++k) {
        const double c = p->molar[k];
        const double h = c > 0.0 ? 1e-3 * c : 1e-9;
        double dex[2][DFT_MAXS] = {}, des[2][DFT_MAXS] = {}, dg[2] = {};
        for (int lev = 0; lev < 2; ++lev) {
            const double hh = lev == 0 ? h : 0.5 * h;
            BathState bp, bm;
            std::vector<double> cp(p->molar), cm(p->molar);
            cp[k] = c + hh;
            cm[k] = c - hh;
            if (cm[k] < 0.0) cm[k] = 0.0;
            const double span = cp[k] - cm[k];
            if (!compute_bath(S, p->R.data(), p->z.data(), cp.data(), p->T, p->eps_r, &bp, err, p->g.phi) ||
                !compute_bath(S, p->R.data(), p->z.data(), cm.data(), p->T, p->eps_r, &bm, err, p->g.phi))
                return false;
            for (int i = 0; i < S; ++i) {
                dex[lev][i] = ((bp.mu_hs[i] + bp.mu_es[i]) - (bm.mu_hs[i] + bm.mu_es[i])) / span;
                des[lev][i] = (bp.mu_es[i] - bm.mu_es[i]) / span;
            }
            dg[lev] = (bp.gamma - bm.gamma) / span;
        }
        for (int i = 0; i < S; ++i) {
            d->dmu_ex[i * S + k] = (4.0 * dex[1][i] - dex[0][i]) / 3.0 / to_rho;
            d->dmu_es[i * S + k] = (4.0 * des[1][i] - des[0][i]) / 3.0 / to_rho;
        }
        d->dgamma[k] = (4.0 * dg[1] - dg[0]) / 3.0 / to_rho;
    }
    return true;
}

// Bulk-fluid kernel at k = 0 (limits of the ball integrals), in kT nm^3
double delta_c_hat_zero(const dft_plan* p, int i, int j) {
    const BathState& b = p->bath;
    const double pi = 3.14159265358979323846;
    const double R = p->R[i] + p->R[j];
    const double pref = 0.5 * b.lb * p->z[i] * p->z[j];
    double a = 0.0, bb = 0.0, c = 2.0;
    if (b.gamma > 0.0) {
        const double li = b.lam[i], lj = b.lam[j];
        a = 1.0 / (2.0 * li * lj);
        bb = (li + lj) / (li * lj);
        c = (li - lj) * (li - lj) / (2.0 * li * lj) + 2.0;
    }
    return pref * (a * pi * R * R * R * R - bb * 4.0 * pi * R * R * R / 3.0 + c * 2.0 * pi * R * R);
}

template <typename Real>
dft_status grad_t(dft_plan* p, const Real* rho, const Real* V, double* omega_out, Real* d_rho, Real* d_V,
                  double* d_bulk) {
    using O = Ops<Real>;
    using P = Passes<Real>;
    const SpeciesDesc<Real>& sp = species<Real>(p);
    const int S = p->S;
    const long long n_zk = ceil_div(p->g.nxh, p->Tz) * p->g.ny;
    const long long n_phi = p->blocks_x(p->LRphi);
    const long long n_g = p->blocks_x(p->LRupd);
    const size_t need = size_t(2 * n_zk + n_phi + n_g * (S + 1));
    if (p->grad_red_len < need) {
        cudaFree(p->grad_red);
        p->grad_red = nullptr;
        if (cudaMalloc(&p->grad_red, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            p->grad_red_len = 0;
            return fail(p, DFT_ENOMEM, "gradient partial sums");
        }
        p->grad_red_len = need;
    }
    double* r_energy = p->grad_red;
    double* r_phi = r_energy + 2 * n_zk;
    double* r_g = r_phi + n_phi;
    const double dv = p->g.hx * p->g.hy * p->g.hz;
    TRY(reset_status(p));
    TRY(O::first_half(p, rho, p->slotA, 0, r_energy));
    TRY(finalize(p, FIN_IDENTITY, 0, 0, -1.0));
    LAUNCH(p, K_XPHI, 2.0 * DFT_NSPEC * CB(p), P::xphi(p->stream, p->g, p->ax, p->LRphi, p->ctl, O::slot_n(p->slotA),
                                                        nullptr, nullptr, O::T1(p), p->red_max, &p->ctl->status,
                                                        r_phi, O::kf(p, 0), O::tw(p, 0)));
    LAUNCH(p, K_YFFT, 2.0 * DFT_NSPEC * CB(p), P::yfft(p->stream, false, p->g, p->ay, p->Ty, DFT_NSPEC, O::T1(p),
                                                        &p->ctl->status, O::tw(p, 1), p->wait_polls));
    LAUNCH(p, K_ZBWD, (DFT_NSPEC + 2 * S) * CB(p),
           P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 3, S, p->ctl,
                        O::T1(p), O::slot_es(p, p->slotA), nullptr, nullptr, O::tw(p, 2)));
    LAUNCH(p, K_YFFT, 2.0 * S * CB(p), P::yfft(p->stream, true, p->g, p->ay, p->Ty, S, O::T1(p), &p->ctl->status,
                                                O::tw(p, 1), p->wait_polls));
    LAUNCH(p, K_XUPD, S * (CB(p) + RB(p) * (2 + (d_rho ? 1 : 0) + (d_V ? 1 : 0))),
           P::xgrad(p->stream, p->g, p->ax, sp, p->LRupd, Real(dv), O::T1(p), rho, V, d_rho, d_V, r_g, O::tw(p, 0)));
    std::vector<double> h(need);
    cudaError_t e = cudaMemcpyAsync(h.data(), p->grad_red, need * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("reading gradient sums: ") + cudaGetErrorString(e));
    if (p->ctl_host->status & DEV_TIMEOUT) return fail(p, DFT_ETIMEOUT, "a bounded wait on an asynchronous copy gave up");
    if (p->ctl_host->status & DEV_N3BOUND) return fail(p, DFT_EN3BOUND, "local packing fraction n3 >= 1 met");
    double energy = 0.0, qgam = 0.0, phisum = 0.0, ideal = 0.0;
    std::vector<double> Ni(S, 0.0);
    for (long long b = 0; b < n_zk; ++b) { energy += h[2 * b]; qgam += h[2 * b + 1]; }
    for (long long b = 0; b < n_phi; ++b) phisum += h[2 * n_zk + b];
    for (long long b = 0; b < n_g; ++b) {
        const double* r = &h[2 * n_zk + n_phi + b * (S + 1)];
        ideal += r[0];
        for (int i = 0; i < S; ++i) Ni[i] += r[1 + i];
    }
    const double N = double(p->g.n);
    const BathState& bt = p->bath;
    std::vector<double> D(S);
    for (int i = 0; i < S; ++i) D[i] = Ni[i] - N * bt.rho[i];
    double lin = 0.0;
    for (int i = 0; i < S; ++i) lin += bt.mu_es[i] * D[i];
    // Omega/kT = h^3 [ideal + ext + sum Phi + sum_i mu_ES_bath_i D_i - (1/2) sum_i sum_x drho_i E_i],
    // sum_x drho_i E_i = (1/N) sum_k conj(drho_hat_i) es_hat_i (Parseval)
    const double omega = dv * (ideal + phisum + lin - 0.5 * energy / N);
    if (!std::isfinite(omega)) return fail(p, DFT_ENONFINITE, "non-finite grand potential");
    if (omega_out) *omega_out = omega;
    if (d_bulk) {
        BathDerivs bd;
        std::string err;
        if (!bath_derivatives(p, &bd, &err)) return fail(p, DFT_EINVAL, err);
        for (int k = 0; k < S; ++k) {
            double g = 0.0;
            if (bt.rho[k] > 0.0) g -= Ni[k] / bt.rho[k];
            for (int i = 0; i < S; ++i) g -= Ni[i] * bd.dmu_ex[i * S + k];
            for (int i = 0; i < S; ++i) g += bd.dmu_es[i * S + k] * D[i];
            g -= bt.mu_es[k] * N;
            g -= 0.5 * bd.dgamma[k] * qgam / N;
            for (int j = 0; j < S; ++j) g += delta_c_hat_zero(p, k, j) * D[j];
            d_bulk[k] = dv * g;
        }
    }
    return DFT_OK;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
namespace {
// --------------------------------------------------------------------------------------
// Newton-Krylov solver (see newton.cu): u = log rho on the accessible voxels,
// F(u) = u - log G(e^u); GMRES(m) on J d = -F with finite-difference products J v, a
// backtracking line search on |F|; stops on the Picard residual r(rho) < tol.
// --------------------------------------------------------------------------------------
template <typename Real>
dft_status newton_t(dft_plan* p, Real* rho, const Real* V, double tol, int max_newton, int m, int* iters_out,
                    int* gevals_out, double* resid_out) {
    const long long n = (long long)p->S * p->g.n;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 2 * sms;
    NkVec<Real> vk(p->stream, n, grid);
    std::vector<Real*> buf;
    auto alloc = [&](size_t count) -> Real* {
        void* q = nullptr;
        if (cudaMalloc(&q, count * sizeof(Real)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        buf.push_back(static_cast<Real*>(q));
        return static_cast<Real*>(q);
    };
    double* part_dev = nullptr;
    std::vector<double> part_host(grid);
    struct Cleanup {
        std::vector<Real*>& b;
        double*& pd;
        ~Cleanup() { for (Real* q : b) cudaFree(q); cudaFree(pd); }
    } cleanup{buf, part_dev};
    Real* F = alloc(n);
    Real* Ft = alloc(n);
    Real* g = alloc(n);
    Real* gt = alloc(n);
    Real* rt = alloc(n);
    Real* d = alloc(n);
    Real* basis = alloc(size_t(m + 1) * n);
    if (!F || !Ft || !g || !gt || !rt || !d || !basis || cudaMalloc(&part_dev, sizeof(double) * grid) != cudaSuccess) {
        cudaGetLastError();
        return fail(p, DFT_ENOMEM, "Newton-Krylov work vectors");
    }
    auto Vk = [&](int i) { return basis + size_t(i) * n; };
    int gevals = 0;
    // G(x) into gout and the Picard residual r(x); a status error (n3 >= 1, non-finite) is returned
    auto evalG = [&](const Real* x, Real* gout, double* r) -> dft_status {
        ++gevals;
        dft_status st = picard_map_t<Real>(p, x, V, gout);
        if (st != DFT_OK) return st;
        st = read_ctl(p);
        if (st != DFT_OK) return st;
        if (r) *r = p->ctl_host->resid;
        return DFT_OK;
    };
    auto dot = [&](const Real* a, const Real* b, double* out) -> dft_status {
        cudaError_t e = vk.dot(a, b, part_dev, part_host.data(), out);
        return e == cudaSuccess ? DFT_OK : fail(p, DFT_ECUDA, std::string("Newton-Krylov: ") + cudaGetErrorString(e));
    };
#define NK_CUDA(x)                                                                                       \
    do {                                                                                                 \
        cudaError_t _e = (x);                                                                            \
        if (_e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("Newton-Krylov: ") + cudaGetErrorString(_e)); \
    } while (0)
    double r = 0.0, fn2 = 0.0;
    TRY(evalG(rho, g, &r));
    NK_CUDA(vk.residual(rho, g, V, F));
    TRY(dot(F, F, &fn2));
    double fn = std::sqrt(fn2);
    const double macheps = sizeof(Real) == 4 ? 1.1920929e-7 : 2.220446049250313e-16;
    const double eps = std::sqrt(macheps) * std::sqrt(double(n));
    const double eta = 0.1;            // GMRES relative tolerance (forcing term)
    std::vector<double> H(size_t(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), gv(m + 1, 0.0), y(m, 0.0);
    int it = 0;
    for (; it < max_newton && !(r < tol) && fn > 0.0; ++it) {
        // GMRES(m) on J d = -F from d = 0
        NK_CUDA(vk.axpby(-1.0 / fn, F, 0.0, Vk(0)));
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = fn;
        int jm = 0;
        for (int j = 0; j < m; ++j) {
            // w = J v_j
            NK_CUDA(vk.step(rho, Vk(j), eps, V, rt));
            TRY(evalG(rt, gt, nullptr));
            NK_CUDA(vk.jv(rt, gt, F, V, eps, Vk(j + 1)));
            for (int i = 0; i <= j; ++i) {      // modified Gram-Schmidt
                double h = 0.0;
                TRY(dot(Vk(j + 1), Vk(i), &h));
                H[size_t(i) * m + j] = h;
                NK_CUDA(vk.axpby(-h, Vk(i), 1.0, Vk(j + 1)));
            }
            double hn2 = 0.0;
            TRY(dot(Vk(j + 1), Vk(j + 1), &hn2));
            const double hn = std::sqrt(hn2);
            H[size_t(j + 1) * m + j] = hn;
            if (hn > 0.0) NK_CUDA(vk.axpby(1.0 / hn, Vk(j + 1), 0.0, Vk(j + 1)));
            for (int i = 0; i < j; ++i) {       // previous rotations on column j
                const double a = H[size_t(i) * m + j], b = H[size_t(i + 1) * m + j];
                H[size_t(i) * m + j] = cs[i] * a + sn[i] * b;
                H[size_t(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[size_t(j) * m + j], b = H[size_t(j + 1) * m + j];
            const double rr = std::hypot(a, b);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? b / rr : 0.0;
            H[size_t(j) * m + j] = rr;
            H[size_t(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            jm = j + 1;
            if (std::fabs(gv[j + 1]) <= eta * fn || hn == 0.0) break;
        }
        for (int i = jm - 1; i >= 0; --i) {     // back substitution
            double t = gv[i];
            for (int k = i + 1; k < jm; ++k) t -= H[size_t(i) * m + k] * y[k];
            y[i] = H[size_t(i) * m + i] != 0.0 ? t / H[size_t(i) * m + i] : 0.0;
        }
        NK_CUDA(vk.axpby(y[0], Vk(0), 0.0, d));
        for (int i = 1; i < jm; ++i) NK_CUDA(vk.axpby(y[i], Vk(i), 1.0, d));
        // backtracking on |F|: u <- u + lam d
        double lam = 1.0, rnew = r, ftn = fn;
        bool accepted = false;
        for (int t = 0; t < 8 && !accepted; ++t, lam *= 0.5) {
            NK_CUDA(vk.step(rho, d, lam, V, rt));
            dft_status st = evalG(rt, gt, &rnew);
            if (st == DFT_EN3BOUND || st == DFT_ENONFINITE) continue;     // too long a step
            if (st != DFT_OK) return st;
            NK_CUDA(vk.residual(rt, gt, V, Ft));
            double f2 = 0.0;
            TRY(dot(Ft, Ft, &f2));
            ftn = std::sqrt(f2);
            if (ftn <= (1.0 - 1e-4 * lam) * fn) accepted = true;
        }
        if (!accepted) break;
        NK_CUDA(cudaMemcpyAsync(rho, rt, sizeof(Real) * n, cudaMemcpyDeviceToDevice, p->stream));
        std::swap(g, gt);
        std::swap(F, Ft);
        fn = ftn;
        r = rnew;
    }
#undef NK_CUDA
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(p, DFT_ECUDA, "Newton-Krylov: synchronize");
    if (iters_out) *iters_out = it;
    if (gevals_out) *gevals_out = gevals;
    if (resid_out) *resid_out = r;
    if (!(r < tol)) return fail(p, DFT_ENOCONV, "Newton-Krylov: tol not reached");
    return DFT_OK;
}
}  // namespace

namespace {
// --------------------------------------------------------------------------------------
// x-pass autotuner: rows per block of the three x passes that stream every iteration
// (xfwd, xphi, xupdate), timed on the plan's own data and cached per grid, species count
// and precision for the life of the process.
// --------------------------------------------------------------------------------------
struct TuneKey {
    int nx, ny, nz, S, prec;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nz, S, prec) < std::tie(o.nx, o.ny, o.nz, o.S, o.prec);
    }
};
std::mutex g_tune_mu;
struct TuneResult {
    std::array<int, 6> lines;       // LX, LRphi, LRupd, LRn3, LRphi2, LRupd2
    int xrt, xpers, yrt, zgrp, zsplit;   // transform variants (GridDesc)
    AxisPlan ax;                    // radix order of the x passes
};
std::map<TuneKey, TuneResult> g_tune_cache;

// Candidate radix orders of a run-time transform of length n: the default plan (3s, other odd
// primes, 16s, then 2/4/8), its reverse, and for powers of two one of 8s (then 4 or 2) and one of
// 4s (then 2).
std::vector<AxisPlan> radix_orders(int n) {
    std::vector<AxisPlan> out;
    AxisPlan d;
    if (!dft_radix_plan(n, &d)) return out;
    out.push_back(d);
    AxisPlan r = d;
    std::reverse(r.radix, r.radix + r.nstages);
    auto same = [](const AxisPlan& a, const AxisPlan& b) {
        if (a.nstages != b.nstages) return false;
        for (int s = 0; s < a.nstages; ++s)
            if (a.radix[s] != b.radix[s]) return false;
        return true;
    };
    auto add = [&](const AxisPlan& a) {
        for (const AxisPlan& o : out)
            if (same(o, a)) return;
        out.push_back(a);
    };
    add(r);
    if ((n & (n - 1)) == 0) {
        for (int big : {8, 4}) {
            AxisPlan q{n, 0, {}};
            int m = n;
            while (m % big == 0 && q.nstages < DFT_MAXSTAGES) { q.radix[q.nstages++] = big; m /= big; }
            if (m > 1 && q.nstages < DFT_MAXSTAGES) q.radix[q.nstages++] = m;
            if (m <= 16 && q.nstages <= DFT_MAXSTAGES) add(q);
        }
    }
    return out;
}

std::string radix_text(const AxisPlan& a) {
    std::string s;
    for (int i = 0; i < a.nstages; ++i) s += (i ? "x" : "") + std::to_string(a.radix[i]);
    return s;
}

std::string ct_radix_text(int n) {
    std::string s;
    for (int i = 0; i < ct_nstages(n); ++i) s += (i ? "x" : "") + std::to_string(ct_radix_at(n, i));
    return s;
}

// Text of a plan's transform variants and rows per block (dft_plan_tuning).
void describe_tuning(dft_plan* p) {
    const GridDesc& g = p->g;
    std::string t = "x: ";
    t += (!g.xrt && dft_is_ct_size(g.nx)) ? "compile-time radix " + ct_radix_text(g.nx)
                                          : "run-time radix " + radix_text(p->ax);
    if (!g.xrt && dft_is_ct_size(g.nx) && g.xpers)
        t += g.xpers == 2 ? ", persistent Phi' passes with cp.async prefetch"
                          : ", persistent Phi' passes with bulk-copy prefetch";
    t += "; rows per block xfwd " + std::to_string(p->LX) + ", xphi " + std::to_string(p->LRphi) + ", xupdate " +
         std::to_string(p->LRupd) + ", n3 max " + std::to_string(p->LRn3) + ", paired xphi " +
         std::to_string(p->LRphi2) + ", paired xupdate " + std::to_string(p->LRupd2);
    t += "; y: ";
    t += (!g.yrt && dft_is_ct_size(g.ny)) ? "TMA persistent, " + std::to_string(p->precision == DFT_FP64 ? 8 : 16) +
                                                "-column tiles"
                                          : "run-time column kernel, " + std::to_string(p->Ty) + "-column tiles";
    t += "; z: ";
    t += dft_is_ct_size(g.nz) ? (g.zgrp ? std::string("grouped, one tile per CTA") : std::string("TMA persistent"))
                              : "run-time column kernel, " + std::to_string(p->Tz) + "-column tiles";
    if (dft_is_ct_size(g.nz) && g.zsplit) t += ", first half as z transforms and a k-space products pass";
    t += p->pdl_on ? "; launches: programmatic dependent" : "; launches: stream order";
    p->tuning = t;
}

template <typename Real> dft_status autotune_t(dft_plan* p, const Real* rho, const Real* V, int reps) {
    using O = Ops<Real>;
    using P = Passes<Real>;
    using C = typename Cplx<Real>::type;
    const SpeciesDesc<Real>& sp = species<Real>(p);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool prof = p->prof;
    p->prof = false;
    // realistic spectra in slot A (weighted densities of rho) and T1
    TRY(reset_status(p));
    TRY(O::first_half(p, rho, p->slotA, 0));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 11, 16};
    // a candidate whose launch is refused (shared memory) is skipped
    auto time_it = [&](auto&& launch) -> float {
        cudaGetLastError();
        launch();   // warm
        if (cudaGetLastError() != cudaSuccess) return 1e30f;
        cudaEventRecord(e0, p->stream);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, p->stream);
        cudaEventSynchronize(e1);
        if (cudaGetLastError() != cudaSuccess) return 1e30f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const int lpr_upd = (p->S + 1) / 2;
    int best[6] = {p->LX, p->LRphi, p->LRupd, p->LRn3, p->LRphi2, p->LRupd2};
    float best_ms[6] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    const C* A = O::slot_n(p->slotA);
    Offsets<Real> off0;
    for (int c = 0; c < DFT_NCOMP + 2; ++c) off0.v[c] = Real(0);
    const int cand_n3[] = {8, 16, 24, 30, 32, 48, 62, 64};
    for (int L : cand_n3) {
        if (P::smem_x(p->g.nx, L) > size_t(optin)) continue;
        const float ms = time_it([&] {
            P::xinv(p->stream, p->g, p->ax, L, 1, A + 3 * p->g.nc, nullptr, nullptr, off0, 0, p->red_max, 0,
                    O::kf(p, 0), O::tw(p, 0));
        });
        if (ms < best_ms[3]) { best_ms[3] = ms; best[3] = L; }
    }
    for (int L : cand) {
        if (P::smem_x(p->g.nx, L) <= size_t(optin)) {
            const float ms = time_it([&] {
                P::xfwd(p->stream, p->g, p->ax, p->S, L, rho, O::T1(p), O::tw(p, 0));
            });
            if (ms < best_ms[0]) { best_ms[0] = ms; best[0] = L; }
        }
        if (P::smem_x(p->g.nx, 5 * L) <= size_t(optin)) {
            const float ms = time_it([&] {
                P::xphi(p->stream, p->g, p->ax, L, p->ctl, A, A, nullptr, O::T1(p), p->red_max, &p->ctl->status,
                        nullptr, O::kf(p, 0), O::tw(p, 0));
            });
            if (ms < best_ms[1]) { best_ms[1] = ms; best[1] = L; }
        }
        if (P::smem_x(p->g.nx, lpr_upd * L) <= size_t(optin)) {
            const float ms = time_it([&] {
                // as in the iteration: the accepted point's pass also writes G's x spectra
                P::xupdate(p->stream, p->g, p->ax, sp, L, p->ctl, O::T1(p), rho, rho, V, nullptr, nullptr,
                           static_cast<C*>(p->gspec), nullptr, p->red_sum, &p->ctl->status, O::tw(p, 0));
            });
            if (ms < best_ms[2]) { best_ms[2] = ms; best[2] = L; }
        }
        // the paired-sample passes (weights of ctl[1], ctl[2]: zero at create, any values time alike)
        if (P::smem_x(p->g.nx, 10 * L) <= size_t(optin)) {
            const float ms = time_it([&] {
                P::xphi2(p->stream, p->g, p->ax, L, p->ctl, A, A, O::T1(p), &p->ctl->status, O::kf(p, 0), O::tw(p, 0));
            });
            if (ms < best_ms[4]) { best_ms[4] = ms; best[4] = L; }
        }
        if (P::smem_x(p->g.nx, 2 * lpr_upd * L) <= size_t(optin)) {
            const float ms = time_it([&] {
                P::xupdate2(p->stream, p->g, p->ax, sp, L, p->ctl, O::T1(p), O::T1(p), rho, rho, V, nullptr,
                            p->red_sum, p->red_sum2, &p->ctl->status, O::tw(p, 0));
            });
            if (ms < best_ms[5]) { best_ms[5] = ms; best[5] = L; }
        }
    }
    p->LX = best[0];
    p->LRphi = best[1];
    p->LRupd = best[2];
    p->LRn3 = best[3];
    p->LRphi2 = best[4];
    p->LRupd2 = best[5];
    // The persistent Phi' passes (compile-time lengths; bulk copies, then cp.async): their own
    // rows per block, kept if the single and paired passes together are faster than the
    // per-block kernels and the other persistent form.
    if (dft_is_ct_size(p->g.nx)) {
        float best_sum = best_ms[1] + best_ms[4];
        int best_pers = 0;
        int bp_best[2] = {p->LRphi, p->LRphi2};
        for (int pers = 1; pers <= 2; ++pers) {
            p->g.xpers = pers;
            int bp[2] = {p->LRphi, p->LRphi2};
            float bpm[2] = {1e30f, 1e30f};
            for (int L : cand) {
                float ms = time_it([&] {
                    P::xphi(p->stream, p->g, p->ax, L, p->ctl, A, A, nullptr, O::T1(p), p->red_max, &p->ctl->status,
                            nullptr, O::kf(p, 0), O::tw(p, 0));
                });
                if (ms < bpm[0]) { bpm[0] = ms; bp[0] = L; }
                ms = time_it([&] {
                    P::xphi2(p->stream, p->g, p->ax, L, p->ctl, A, A, O::T1(p), &p->ctl->status, O::kf(p, 0),
                             O::tw(p, 0));
                });
                if (ms < bpm[1]) { bpm[1] = ms; bp[1] = L; }
            }
            if (bpm[0] + bpm[1] < best_sum) {
                best_sum = bpm[0] + bpm[1];
                best_pers = pers;
                bp_best[0] = bp[0];
                bp_best[1] = bp[1];
            }
        }
        p->g.xpers = best_pers;
        if (best_pers) {
            p->LRphi = bp_best[0];
            p->LRphi2 = bp_best[1];
        }
    }
    // Transform variants, timed on the same data with the rows per block just chosen.
    // x: the compile-time Phi' pass (where the length has one) against the run-time one under
    // each candidate radix order.
    {
        const AxisPlan ax0 = p->ax;
        float bms = 1e30f;
        int bxrt = 1;
        AxisPlan bax = ax0;
        auto time_xphi = [&] {
            return time_it([&] {
                P::xphi(p->stream, p->g, p->ax, p->LRphi, p->ctl, A, A, nullptr, O::T1(p), p->red_max,
                        &p->ctl->status, nullptr, O::kf(p, 0), O::tw(p, 0));
            });
        };
        if (dft_is_ct_size(p->g.nx)) {
            p->g.xrt = 0;
            bms = time_xphi();
            bxrt = 0;
        }
        for (const AxisPlan& o : radix_orders(p->g.nx)) {
            if (P::smem_x(p->g.nx, 5 * p->LRphi) > size_t(optin)) break;
            p->g.xrt = 1;
            p->ax = o;
            const float ms = time_xphi();
            if (ms < bms) { bms = ms; bxrt = 1; bax = o; }
        }
        p->g.xrt = bxrt;
        p->ax = bxrt ? bax : ax0;
    }
    // y: the persistent TMA pass against the run-time column kernel (nine components forward)
    if (dft_is_ct_size(p->g.ny)) {
        float ms[2];
        for (int v = 0; v < 2; ++v) {
            p->g.yrt = v;
            ms[v] = time_it([&] {
                P::yfft(p->stream, false, p->g, p->ay, p->Ty, DFT_NSPEC, O::T1(p), &p->ctl->status, O::tw(p, 1),
                        p->wait_polls);
            });
        }
        p->g.yrt = ms[1] < ms[0] ? 1 : 0;
    }
    // z: the persistent TMA passes against the grouped one-tile-per-CTA kernels (both halves)
    if (dft_is_ct_size(p->g.nz)) {
        float ms[2];
        for (int v = 0; v < 2; ++v) {
            p->g.zgrp = v;
            ms[v] = time_it([&] {
                P::zconv_fwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 0, O::T1(p),
                             O::slot_n(p->slotB), O::slot_es(p, p->slotB), nullptr, O::tw(p, 2), &p->ctl->status);
                P::zconv_bwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 3, p->S,
                             p->ctl, O::T1(p), O::slot_es(p, p->slotA), O::slot_es(p, p->slotB), nullptr,
                             O::tw(p, 2));
            });
        }
        p->g.zgrp = ms[1] < ms[0] ? 1 : 0;
        // the first-half z stage as one pass (the choice above) or split into z transforms and a
        // k-space products pass; the two often time within a few per cent, so each is timed in
        // four alternating rounds and its best round counts
        auto stage_z = [&](int v) {
            p->g.zsplit = v;
            if (v) {
                P::zfft(p->stream, false, p->g, p->S, O::T1(p), &p->ctl->status, O::tw(p, 2), p->wait_polls);
                P::zmul(p->stream, p->g, sp, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), O::T1(p), O::slot_n(p->slotB),
                        O::slot_es(p, p->slotB));
                P::zfft(p->stream, true, p->g, DFT_NSPEC, O::slot_n(p->slotB), &p->ctl->status, O::tw(p, 2),
                        p->wait_polls);
            } else {
                P::zconv_fwd(p->stream, p->g, p->az, sp, p->Tz, O::kf(p, 0), O::kf(p, 1), O::kf(p, 2), 0, O::T1(p),
                             O::slot_n(p->slotB), O::slot_es(p, p->slotB), nullptr, O::tw(p, 2), &p->ctl->status);
            }
        };
        float best_v[2] = {1e30f, 1e30f};
        for (int round = 0; round < 4; ++round) {
            for (int v = 0; v < 2; ++v) {
                const float t = time_it([&] { stage_z(v); });
                if (t < best_v[v]) best_v[v] = t;
            }
        }
        p->g.zsplit = best_v[1] < best_v[0] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaStreamSynchronize(p->stream);
    p->prof = prof;
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    TRY(reset_status(p));
    return DFT_OK;
}
}  // namespace

namespace {
void release_iter_graph(dft_plan* p) {
    if (p->iexec) cudaGraphExecDestroy(p->iexec);
    if (p->igraph) cudaGraphDestroy(p->igraph);
    p->iexec = nullptr;
    p->igraph = nullptr;
    p->iloop = false;
}

// On-device iteration loop: a graph whose only node is a conditional WHILE node; its body is one
// iteration followed by k_loop_tail, which counts the iterations left (set by k_loop_set before
// each launch) and clears the condition after the last, so one graph launch runs all of them
// without returning to the host.
__global__ void k_loop_set(int* left, int n) { *left = n; }
__global__ void k_loop_tail(cudaGraphConditionalHandle h, int* left) {
    const int n = *left - 1;
    *left = n;
    cudaGraphSetConditional(h, n > 0 ? 1u : 0u);
}

// Build the loop graph: `body` queues one iteration on `st` (a capture stream) and returns a
// status.  On success *graph holds the loop; a runtime without conditional nodes returns an
// error and the caller replays a one-iteration graph instead.
template <typename F>
cudaError_t build_loop_graph(cudaStream_t st, int* left, cudaGraph_t* graph, dft_status* body_status, F&& body) {
    *graph = nullptr;
    *body_status = DFT_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return e;
    }
    *body_status = body();
    k_loop_tail<<<1, 1, 0, st>>>(h, left);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(st, &captured);
    if (e == cudaSuccess && *body_status != DFT_OK) e = cudaErrorUnknown;
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return e;
    }
    *graph = g;
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* dft_version(void) { return "gb300dft 0.1 (sm_103a)"; }

const char* dft_last_error(const dft_plan* plan) {
    return plan ? plan->err.c_str() : g_create_error.c_str();
}

dft_status dft_plan_create(const dft_params* prm, void* cuda_stream, dft_plan** out) {
    if (!prm || !out) return fail(nullptr, DFT_EINVAL, "NULL params or out");
    *out = nullptr;
    if (!dft_valid_length(prm->nx) || !dft_valid_length(prm->ny) || !dft_valid_length(prm->nz))
        return fail(nullptr, DFT_EINVAL, "grid sizes must be 4 <= n <= 512 with prime factors <= 31");
    if (!(prm->hx > 0 && prm->hy > 0 && prm->hz > 0)) return fail(nullptr, DFT_EINVAL, "grid spacing must be > 0");
    if (prm->nspecies < 1 || prm->nspecies > DFT_MAX_SPECIES) return fail(nullptr, DFT_EINVAL, "nspecies out of range");
    if (!prm->radius_nm || !prm->valence || !prm->bulk_molar) return fail(nullptr, DFT_EINVAL, "NULL species array");
    if (!(prm->temperature_K > 0 && prm->eps_r > 0)) return fail(nullptr, DFT_EINVAL, "T and eps_r must be > 0");
    if (prm->precision != DFT_FP32_STAB && prm->precision != DFT_FP64)
        return fail(nullptr, DFT_EINVAL, "unknown precision");
    const int S = prm->nspecies;
    double charge = 0.0, scale = 0.0, eta = 0.0;
    for (int i = 0; i < S; ++i) {
        if (!(prm->radius_nm[i] > 0)) return fail(nullptr, DFT_EINVAL, "radius must be > 0");
        if (!(prm->bulk_molar[i] >= 0)) return fail(nullptr, DFT_EINVAL, "bulk concentration must be >= 0");
        charge += prm->valence[i] * prm->bulk_molar[i];
        scale += std::fabs(prm->valence[i]) * prm->bulk_molar[i];
        eta += prm->bulk_molar[i] * 0.602214076 * 4.18879020478639098 * std::pow(prm->radius_nm[i], 3);
    }
    if (std::fabs(charge) > 1e-12 * scale) return fail(nullptr, DFT_ENONNEUTRAL, "bath is not electroneutral");
    if (eta >= kN3Bound) return fail(nullptr, DFT_EINVAL, "bath packing fraction >= 0.9");

    dft_plan* p = new dft_plan();
    p->S = S;
    p->precision = prm->precision;
    p->R.assign(prm->radius_nm, prm->radius_nm + S);
    p->z.assign(prm->valence, prm->valence + S);
    p->molar.assign(prm->bulk_molar, prm->bulk_molar + S);
    p->n_fixed.assign(S, 0.0);
    if (prm->n_fixed)
        for (int i = 0; i < S; ++i) {
            if (!(prm->n_fixed[i] >= 0.0)) {
                delete p;
                return fail(nullptr, DFT_EINVAL, "n_fixed must be >= 0");
            }
            p->n_fixed[i] = prm->n_fixed[i];
            if (p->n_fixed[i] > 0.0) p->ncanon += 1;
        }
    p->T = prm->temperature_K;
    p->eps_r = prm->eps_r;
    if (prm->functional != DFT_PHI_RSLT && prm->functional != DFT_PHI_ROSENFELD &&
        prm->functional != DFT_PHI_WHITE_BEAR) {
        delete p;
        return fail(nullptr, DFT_EINVAL, "unknown functional");
    }
    std::string err;
    if (!compute_bath(S, p->R.data(), p->z.data(), p->molar.data(), p->T, p->eps_r, &p->bath, &err,
                      prm->functional)) {
        delete p;
        return fail(nullptr, DFT_EINVAL, err);
    }
    GridDesc& g = p->g;
    g.phi = prm->functional;
    g.nx = prm->nx; g.ny = prm->ny; g.nz = prm->nz;
    g.nxh = g.nx / 2 + 1;
    g.pxh = (g.nxh + 1) & ~1;
    g.n = (long long)g.nx * g.ny * g.nz;
    g.nc = (long long)g.nz * g.ny * g.pxh;
    g.hx = prm->hx; g.hy = prm->hy; g.hz = prm->hz;
    g.pdl = 1;
    const double two_pi = 6.28318530717958647692;
    p->kf[0] = two_pi / (g.nx * g.hx);
    p->kf[1] = two_pi / (g.ny * g.hy);
    p->kf[2] = two_pi / (g.nz * g.hz);
    if (!dft_radix_plan(g.nx, &p->ax) || !dft_radix_plan(g.ny, &p->ay) || !dft_radix_plan(g.nz, &p->az)) {
        delete p;
        return fail(nullptr, DFT_EINVAL, "no radix plan for the grid sizes");
    }
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&p->device);
    const bool f64 = prm->precision == DFT_FP64;
    p->csize = f64 ? sizeof(double2) : sizeof(float2);
    p->rsize = f64 ? sizeof(double) : sizeof(float);
    p->Ty = f64 ? Passes<double>::tile_y(g.ny, 100 * 1024) : Passes<float>::tile_y(g.ny, 100 * 1024);
    p->Tz = f64 ? Passes<double>::tile_z(g.nz, 112 * 1024) : Passes<float>::tile_z(g.nz, 112 * 1024);
    {   // run-time lengths: narrower column tiles while a column pass would have fewer than two
        // CTAs per SM (small grids)
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || sms < 1) sms = 1;
        if (!dft_is_ct_size(g.ny))
            while (p->Ty > 1 && ceil_div(g.nxh, p->Ty) * g.nz < 2LL * sms) p->Ty /= 2;
        if (!dft_is_ct_size(g.nz))
            while (p->Tz > 1 && ceil_div(g.nxh, p->Tz) * g.ny < 2LL * sms) p->Tz /= 2;
    }
    p->LX = pick_lines(g.nx, p->csize, 1, env_budget("DFT_XFWD_SMEM", 48 * 1024), 32);
    p->LRphi = pick_lines(g.nx, p->csize, 5, env_budget("DFT_XPHI_SMEM", 32 * 1024), 16);
    p->LRupd = pick_lines(g.nx, p->csize, (S + 1) / 2, env_budget("DFT_XUPD_SMEM", 48 * 1024), 16);
    p->LRphi2 = pick_lines(g.nx, p->csize, 10, env_budget("DFT_XPHI_SMEM", 32 * 1024), 16);
    p->LRupd2 = pick_lines(g.nx, p->csize, 2 * ((S + 1) / 2), env_budget("DFT_XUPD_SMEM", 48 * 1024), 16);
    if (f64) fill_species<double>(p);
    else fill_species<float>(p);

    cudaError_t e = f64 ? Passes<double>::init_attributes() : Passes<float>::init_attributes();
    if (e != cudaSuccess) {
        delete p;
        return fail(nullptr, DFT_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    // twiddles
    const int ns[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        size_t bytes = size_t(ns[a]) * p->csize;
        if (cudaMalloc(&p->tw[a], bytes) != cudaSuccess) { dft_plan_destroy(p); return fail(nullptr, DFT_ENOMEM, "twiddles"); }
        if (f64) {
            std::vector<double2> t;
            fill_twiddles(ns[a], &t);
            cudaMemcpy(p->tw[a], t.data(), bytes, cudaMemcpyHostToDevice);
        } else {
            std::vector<float2> t;
            fill_twiddles(ns[a], &t);
            cudaMemcpy(p->tw[a], t.data(), bytes, cudaMemcpyHostToDevice);
        }
    }
    const size_t slot_comps = DFT_NSPEC + S + 1;
    const size_t nred = size_t(g.ny) * g.nz + 1;
    struct { void** ptr; size_t bytes; const char* what; } allocs[] = {
        // the weighted-density rows (ten) or the two line-search samples' Phi' spectra (2 x nine)
        {&p->T1, size_t(2 * DFT_NSPEC > DFT_NCOMP ? 2 * DFT_NSPEC : DFT_NCOMP) * g.nc * p->csize, "work spectra"},
        {&p->slotA, slot_comps * g.nc * p->csize, "slot A"},
        {&p->slotB, slot_comps * g.nc * p->csize, "slot B"},
        {&p->gbuf, size_t(S) * g.n * p->rsize, "G buffer"},
        {&p->gspec, size_t(S) * g.nc * p->csize, "G spectra"},
        // FP32 iterations carry the iterate as the caller's field plus this low part
        {f64 ? nullptr : &p->rho_lo, size_t(S) * g.n * p->rsize, "iterate low part"},
        {(void**)&p->red_sum, nred * sizeof(double), "reduction sums"},
        {(void**)&p->red_sum2, nred * sizeof(double), "second sample's reduction sums"},
        {(void**)&p->red_max, nred * sizeof(float), "reduction maxima"},
        // the iteration's control block and the two line-search samples' weights
        {(void**)&p->ctl, 3 * sizeof(Ctl), "control blocks"},
    };
    for (auto& a : allocs) {
        if (!a.ptr) continue;
        if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            dft_plan_destroy(p);
            return fail(nullptr, DFT_ENOMEM, std::string("cudaMalloc failed: ") + a.what);
        }
    }
    cudaMemset(p->ctl, 0, 3 * sizeof(Ctl));
    if (p->ncanon > 0 &&
        cudaMalloc(&p->red_canon, (size_t(g.ny) * g.nz + 1) * DFT_MAXS * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        dft_plan_destroy(p);
        return fail(nullptr, DFT_ENOMEM, "cudaMalloc failed: normalisation sums");
    }
    // On a cubic box |k| = kf sqrt(mx^2 + my^2 + mz^2) takes one value per integer m2, so the
    // compile-time z passes read the FMT weights and bulk-fluid kernels from per-m2 tables
    // instead of evaluating them at every point.
    if (dft_is_ct_size(g.nz) && p->kf[0] == p->kf[1] && p->kf[1] == p->kf[2]) {
        const long long m2max = (long long)(g.nx / 2) * (g.nx / 2) + (long long)(g.ny / 2) * (g.ny / 2) +
                                (long long)(g.nz / 2) * (g.nz / 2);
        const long long P = (long long)S * (S + 1) / 2;
        const long long rows = m2max + 1;
        // records padded to 16 bytes (read with 16-byte loads)
        const long long V = 16 / (long long)p->rsize;
        const long long ws = (2 * S + V - 1) / V * V, ks = (P + V - 1) / V * V;
        if (cudaMalloc(&p->ktab, size_t(rows * (ws + 2 * ks)) * p->rsize) != cudaSuccess) {
            cudaGetLastError();
            dft_plan_destroy(p);
            return fail(nullptr, DFT_ENOMEM, "cudaMalloc failed: |k| tables");
        }
        cudaError_t te;
        if (f64) {
            SpeciesDesc<double>& sp = p->spd;
            double* base = static_cast<double*>(p->ktab);
            sp.tab_w = base; sp.tab_k = base + rows * ws; sp.tab_dk = base + rows * (ws + ks);
            sp.tab_m2max = (int)m2max;
            sp.tab_ws = (int)ws; sp.tab_ks = (int)ks;
            te = Passes<double>::build_ktab(nullptr, sp, p->kf[0]);
        } else {
            SpeciesDesc<float>& sp = p->spf;
            float* base = static_cast<float*>(p->ktab);
            sp.tab_w = base; sp.tab_k = base + rows * ws; sp.tab_dk = base + rows * (ws + ks);
            sp.tab_m2max = (int)m2max;
            sp.tab_ws = (int)ws; sp.tab_ks = (int)ks;
            te = Passes<float>::build_ktab(nullptr, sp, p->kf[0]);
        }
        if (te != cudaSuccess) {
            dft_plan_destroy(p);
            return fail(nullptr, DFT_ECUDA, std::string("|k| tables: ") + cudaGetErrorString(te));
        }
    }
    // The Poisson kernel's lap(k) is a sum of one term per axis: tabulated by FFT index once, with
    // the expression the z passes would evaluate at every point.
    {
        const size_t nl = size_t(g.nx) + g.ny + g.nz;
        if (cudaMalloc(&p->laptab, nl * p->rsize) != cudaSuccess) {
            cudaGetLastError();
            dft_plan_destroy(p);
            return fail(nullptr, DFT_ENOMEM, "cudaMalloc failed: Laplacian table");
        }
        cudaError_t te;
        if (f64) {
            p->spd.lap1d = static_cast<const double*>(p->laptab);
            te = Passes<double>::build_laptab(nullptr, g, p->kf[0], p->kf[1], p->kf[2], static_cast<double*>(p->laptab));
        } else {
            p->spf.lap1d = static_cast<const float*>(p->laptab);
            te = Passes<float>::build_laptab(nullptr, g, float(p->kf[0]), float(p->kf[1]), float(p->kf[2]),
                                             static_cast<float*>(p->laptab));
        }
        if (te != cudaSuccess) {
            dft_plan_destroy(p);
            return fail(nullptr, DFT_ECUDA, std::string("Laplacian table: ") + cudaGetErrorString(te));
        }
    }
    if (cudaMallocHost(&p->ctl_host, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        dft_plan_destroy(p);
        return fail(nullptr, DFT_ENOMEM, "pinned control block");
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dft_plan_destroy(p);
        return fail(nullptr, DFT_ECUDA, std::string("plan setup: ") + cudaGetErrorString(e));
    }
    describe_tuning(p);
    *out = p;
    return DFT_OK;
}

dft_status dft_plan_destroy(dft_plan* p) {
    if (!p) return DFT_OK;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (int a = 0; a < 3; ++a) cudaFree(p->tw[a]);
    cudaFree(p->T1);
    cudaFree(p->slotA);
    cudaFree(p->slotB);
    cudaFree(p->gbuf);
    cudaFree(p->gspec);
    cudaFree(p->rho_lo);
    cudaFree(p->stage_rho);
    cudaFree(p->stage_V);
    cudaFree(p->red_sum);
    cudaFree(p->red_sum2);
    cudaFree(p->red_max);
    cudaFree(p->grad_red);
    cudaFree(p->ktab);
    cudaFree(p->laptab);
    cudaFree(p->red_canon);
    release_iter_graph(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->v_ready) cudaEventDestroy(p->v_ready);
    if (p->side) cudaStreamDestroy(p->side);
    cudaFree(p->ctl);
    if (p->ctl_host) cudaFreeHost(p->ctl_host);
    for (cudaEvent_t ev : p->evpool) cudaEventDestroy(ev);
    delete p;
    return DFT_OK;
}

dft_status dft_plan_bulk(const dft_plan* p, double* rho_bulk, double* mu_hs, double* mu_es, double* gamma,
                         double* beta_p, double* lambda_b) {
    if (!p) return fail(nullptr, DFT_EINVAL, "NULL plan");
    for (int i = 0; i < p->S; ++i) {
        if (rho_bulk) rho_bulk[i] = p->bath.rho[i];
        if (mu_hs) mu_hs[i] = p->bath.mu_hs[i];
        if (mu_es) mu_es[i] = p->bath.mu_es[i];
    }
    if (gamma) *gamma = p->bath.gamma;
    if (beta_p) *beta_p = p->bath.beta_p;
    if (lambda_b) *lambda_b = p->bath.lb;
    return DFT_OK;
}

dft_status dft_weighted_densities(dft_plan* p, const void* rho, void* n_out) {
    TRY(check_plan(p));
    if (!rho || !n_out) return fail(p, DFT_EINVAL, "NULL field pointer");
    p->iter_ready = false;
    if (is_fp64(p)) {
        using O = Ops<double>;
        TRY(O::first_half(p, static_cast<const double*>(rho), p->slotA, 0));
        TRY(O::xinv(p, DFT_NCOMP, O::slot_n(p->slotA), static_cast<double*>(n_out), nullptr, nullptr, -1, nullptr, nullptr));
    } else {
        using O = Ops<float>;
        TRY(O::first_half(p, static_cast<const float*>(rho), p->slotA, 0));
        TRY(O::xinv(p, DFT_NCOMP, O::slot_n(p->slotA), static_cast<float*>(n_out), nullptr, nullptr, -1, nullptr, nullptr));
    }
    return DFT_OK;
}


dft_status dft_c1_hs(dft_plan* p, const void* rho, void* c1_out) {
    TRY(check_plan(p));
    if (!rho || !c1_out) return fail(p, DFT_EINVAL, "NULL field pointer");
    p->iter_ready = false;
    TRY(reset_status(p));
    if (is_fp64(p)) return c1_hs_t<double>(p, static_cast<const double*>(rho), static_cast<double*>(c1_out));
    return c1_hs_t<float>(p, static_cast<const float*>(rho), static_cast<float*>(c1_out));
}


dft_status dft_c1_es(dft_plan* p, const void* rho, void* c1_out, void* psi_out) {
    TRY(check_plan(p));
    if (!rho || !c1_out) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (psi_out && p->S > DFT_MAX_SPECIES - 1) return fail(p, DFT_EINVAL, "psi_out needs nspecies <= 4");
    p->iter_ready = false;
    if (is_fp64(p))
        return c1_es_t<double>(p, static_cast<const double*>(rho), static_cast<double*>(c1_out),
                               static_cast<double*>(psi_out));
    return c1_es_t<float>(p, static_cast<const float*>(rho), static_cast<float*>(c1_out), static_cast<float*>(psi_out));
}


dft_status dft_picard_map(dft_plan* p, const void* rho, const void* V, void* g_out, double* resid_out) {
    TRY(check_plan(p));
    if (!rho || !V || !g_out) return fail(p, DFT_EINVAL, "NULL field pointer");
    p->iter_ready = false;
    if (is_fp64(p))
        TRY(picard_map_t<double>(p, static_cast<const double*>(rho), static_cast<const double*>(V),
                                 static_cast<double*>(g_out)));
    else
        TRY(picard_map_t<float>(p, static_cast<const float*>(rho), static_cast<const float*>(V),
                                static_cast<float*>(g_out)));
    if (resid_out) {
        TRY(read_ctl(p));
        *resid_out = p->ctl_host->resid;
    }
    return DFT_OK;
}

dft_status dft_iter_begin(dft_plan* p, void* rho, const void* V) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    release_iter_graph(p);
    if (is_fp64(p)) return iter_begin_t<double>(p, static_cast<double*>(rho), static_cast<const double*>(V));
    return iter_begin_t<float>(p, static_cast<float*>(rho), static_cast<const float*>(V));
}

dft_status dft_iter_step(dft_plan* p, void* rho, const void* V, double alpha, double* resid_out, double* alpha_out) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (!p->iter_ready || p->iter_rho != rho || p->iter_V != V)
        return fail(p, DFT_EINVAL, "dft_iter_step needs a preceding dft_iter_begin on the same rho and V");
    if (is_fp64(p)) TRY(iter_step_t<double>(p, static_cast<double*>(rho), static_cast<const double*>(V), alpha));
    else TRY(iter_step_t<float>(p, static_cast<float*>(rho), static_cast<const float*>(V), alpha));
    if (resid_out || alpha_out) {
        TRY(read_ctl(p));
        if (resid_out) *resid_out = p->ctl_host->resid_prev;
        if (alpha_out) *alpha_out = p->ctl_host->alpha;
    }
    return DFT_OK;
}

dft_status dft_iter_run(dft_plan* p, void* rho, const void* V, int iters, double alpha, double* resid_out) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (iters < 0) return fail(p, DFT_EINVAL, "negative iteration count");
    if (!p->iter_ready || p->iter_rho != rho || p->iter_V != V)
        return fail(p, DFT_EINVAL, "dft_iter_run needs a preceding dft_iter_begin on the same rho and V");
    if (p->prof) {
        for (int it = 0; it < iters; ++it) TRY(dft_iter_step(p, rho, V, alpha, nullptr, nullptr));
    } else {
        if (p->iexec && (p->graph_rho != rho || p->graph_V != V || p->graph_alpha != alpha)) release_iter_graph(p);
        if (!p->iexec && iters > 0) {
            if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
                return fail(p, DFT_ECUDA, "capture stream creation failed");
            cudaStream_t user = p->stream;
            auto one_iteration = [&]() -> dft_status {
                return is_fp64(p)
                    ? iter_step_t<double>(p, static_cast<double*>(rho), static_cast<const double*>(V), alpha)
                    : iter_step_t<float>(p, static_cast<float*>(rho), static_cast<const float*>(V), alpha);
            };
            // the on-device loop first; a runtime without conditional graph nodes falls back to
            // replays of a one-iteration graph
            p->stream = p->cap;
            cudaGraph_t g = nullptr;
            dft_status st = DFT_OK;
            const int pdl = p->g.pdl;
            cudaError_t e = build_loop_graph(p->cap, &p->ctl->loop_left, &g, &st, one_iteration);
            if ((e != cudaSuccess || st != DFT_OK) && pdl) {
                // a runtime that does not capture programmatic edges: the iteration in stream order
                p->g.pdl = 0;
                st = DFT_OK;
                e = build_loop_graph(p->cap, &p->ctl->loop_left, &g, &st, one_iteration);
            }
            p->stream = user;
            if (st != DFT_OK) {
                p->g.pdl = pdl;
                return st;
            }
            if (e == cudaSuccess) {
                p->iloop = true;
            } else {
                p->stream = p->cap;
                e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) {
                    p->stream = user;
                    p->g.pdl = pdl;
                    return fail(p, DFT_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
                }
                st = one_iteration();
                e = cudaStreamEndCapture(p->cap, &g);
                p->stream = user;
                p->g.pdl = pdl;
                if (st != DFT_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
                p->iloop = false;
            }
            p->g.pdl = pdl;
            p->igraph = g;
            e = cudaGraphInstantiate(&p->iexec, p->igraph, 0);
            if (e != cudaSuccess) {
                release_iter_graph(p);
                return fail(p, DFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            }
            p->graph_rho = rho;
            p->graph_V = V;
            p->graph_alpha = alpha;
        }
        if (p->iloop && iters > 0) {
            k_loop_set<<<1, 1, 0, p->stream>>>(&p->ctl->loop_left, iters);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaGraphLaunch(p->iexec, p->stream);
            if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        } else {
            for (int it = 0; it < iters; ++it) {
                cudaError_t e = cudaGraphLaunch(p->iexec, p->stream);
                if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            }
        }
    }
    if (resid_out) {
        TRY(read_ctl(p));
        *resid_out = p->ctl_host->resid;
    }
    return DFT_OK;
}

dft_status dft_autotune(dft_plan* p, const void* rho, const void* V, int reps, int lines_out[3]) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (reps < 1) reps = 5;
    const TuneKey key{p->g.nx, p->g.ny, p->g.nz, p->S, p->precision};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const TuneResult& t = it->second;
            p->LX = t.lines[0];
            p->LRphi = t.lines[1];
            p->LRupd = t.lines[2];
            p->LRn3 = t.lines[3];
            p->LRphi2 = t.lines[4];
            p->LRupd2 = t.lines[5];
            p->g.xrt = t.xrt;
            p->g.xpers = t.xpers;
            p->g.yrt = t.yrt;
            p->g.zgrp = t.zgrp;
            p->g.zsplit = t.zsplit;
            p->ax = t.ax;
            cached = true;
        }
    }
    if (!cached) {
        if (is_fp64(p)) TRY(autotune_t<double>(p, static_cast<const double*>(rho), static_cast<const double*>(V), reps));
        else TRY(autotune_t<float>(p, static_cast<const float*>(rho), static_cast<const float*>(V), reps));
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneResult{{p->LX, p->LRphi, p->LRupd, p->LRn3, p->LRphi2, p->LRupd2},
                                       p->g.xrt, p->g.xpers, p->g.yrt, p->g.zgrp, p->g.zsplit, p->ax};
    }
    // the iteration state and its graph depend on the block counts and variants
    p->iter_ready = false;
    release_iter_graph(p);
    describe_tuning(p);
    if (lines_out) {
        lines_out[0] = p->LX;
        lines_out[1] = p->LRphi;
        lines_out[2] = p->LRupd;
    }
    return DFT_OK;
}

dft_status dft_picard_step(dft_plan* p, void* rho, const void* V, double alpha, double* resid_out, double* alpha_out) {
    TRY(dft_iter_begin(p, rho, V));
    return dft_iter_step(p, rho, V, alpha, resid_out, alpha_out);
}

dft_status dft_solve_newton(dft_plan* p, void* rho, const void* V, double tol, int max_newton, int krylov_dim,
                            int* newton_out, int* gevals_out, double* resid_out) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (max_newton < 0 || krylov_dim < 1 || krylov_dim > 200) return fail(p, DFT_EINVAL, "bad Newton-Krylov sizes");
    p->iter_ready = false;
    release_iter_graph(p);
    if (is_fp64(p))
        return newton_t<double>(p, static_cast<double*>(rho), static_cast<const double*>(V), tol, max_newton,
                                krylov_dim, newton_out, gevals_out, resid_out);
    return newton_t<float>(p, static_cast<float*>(rho), static_cast<const float*>(V), tol, max_newton, krylov_dim,
                           newton_out, gevals_out, resid_out);
}

dft_status dft_solve(dft_plan* p, void* rho, const void* V, double alpha, double tol, int max_it, int* iters_out,
                     double* resid_out) {
    TRY(dft_iter_begin(p, rho, V));
    TRY(read_ctl(p));
    double r = p->ctl_host->resid;
    int it = 0;
    while (it < max_it && !(r < tol)) {
        // one iteration as a replay of the plan's one-iteration graph, then its residual
        TRY(dft_iter_run(p, rho, V, 1, alpha, &r));
        ++it;
    }
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = r;
    if (!(r < tol)) return fail(p, DFT_ENOCONV, "max_it reached before tol");
    return DFT_OK;
}

dft_status dft_picard_step_host(dft_plan* p, void* rho_host, const void* V_host, double alpha, double* resid_out,
                                double* alpha_out) {
    TRY(check_plan(p));
    if (!rho_host || !V_host) return fail(p, DFT_EINVAL, "NULL host pointer");
    const size_t bytes = size_t(p->S) * p->g.n * p->rsize;
    if (!p->stage_rho) {
        if (cudaMalloc(&p->stage_rho, bytes) != cudaSuccess || cudaMalloc(&p->stage_V, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(p, DFT_ENOMEM, "staging buffers");
        }
    }
    if (!p->side && cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess)
        return fail(p, DFT_ECUDA, "side stream creation failed");
    if (!p->v_ready && cudaEventCreateWithFlags(&p->v_ready, cudaEventDisableTiming) != cudaSuccess)
        return fail(p, DFT_ECUDA, "event creation failed");
    // rho in on the plan's stream; V in on a side stream, awaited only by the first pass that
    // reads it (the first half of G runs meanwhile)
    cudaError_t e = cudaMemcpyAsync(p->stage_rho, rho_host, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->v_ready, p->stream);       // V may be overwritten only now
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->v_ready, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->stage_V, V_host, bytes, cudaMemcpyHostToDevice, p->side);
    if (e == cudaSuccess) e = cudaEventRecord(p->v_ready, p->side);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("H2D copy: ") + cudaGetErrorString(e));
    if (is_fp64(p)) TRY(iter_begin_t<double>(p, static_cast<double*>(p->stage_rho), static_cast<const double*>(p->stage_V), p->v_ready));
    else TRY(iter_begin_t<float>(p, static_cast<float*>(p->stage_rho), static_cast<const float*>(p->stage_V), p->v_ready));
    p->iter_ready = true;
    p->iter_rho = p->stage_rho;
    p->iter_V = p->stage_V;
    // the step as a replay of the cached one-iteration graph, then the control block and rho
    // out with one synchronisation
    TRY(dft_iter_run(p, p->stage_rho, p->stage_V, 1, alpha, nullptr));
    e = cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho_host, p->stage_rho, bytes, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(p, DFT_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(e));
    // a timeout first: the passes after it ran on unfinished spectra
    if (p->ctl_host->status & DEV_TIMEOUT) return fail(p, DFT_ETIMEOUT, "a bounded wait on an asynchronous copy gave up");
    if (p->ctl_host->status & DEV_N3BOUND) return fail(p, DFT_EN3BOUND, "local packing fraction n3 >= 1 met");
    if (p->ctl_host->status & DEV_NONFINITE) return fail(p, DFT_ENONFINITE, "non-finite density or residual met");
    if (resid_out) *resid_out = p->ctl_host->resid_prev;
    if (alpha_out) *alpha_out = p->ctl_host->alpha;
    return DFT_OK;
}

dft_status dft_grad(dft_plan* p, const void* rho, const void* V, double* omega_out, void* dOmega_drho,
                    void* dOmega_dV, double* dOmega_dbulk) {
    TRY(check_plan(p));
    if (!rho || !V) return fail(p, DFT_EINVAL, "NULL field pointer");
    if (p->ncanon > 0) return fail(p, DFT_EINVAL, "dft_grad: the plan has fixed-number species");
    p->iter_ready = false;
    if (is_fp64(p))
        return grad_t<double>(p, static_cast<const double*>(rho), static_cast<const double*>(V), omega_out,
                              static_cast<double*>(dOmega_drho), static_cast<double*>(dOmega_dV), dOmega_dbulk);
    return grad_t<float>(p, static_cast<const float*>(rho), static_cast<const float*>(V), omega_out,
                         static_cast<float*>(dOmega_drho), static_cast<float*>(dOmega_dV), dOmega_dbulk);
}

// ---------------------------------------------------------------------------------------
// Batched state points
// ---------------------------------------------------------------------------------------
}  // extern "C"

struct dft_batch {
    std::vector<dft_plan*> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t main = nullptr;
    bool own_main = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double graph_alpha = 0.0;
    bool loop = false;              // the graph is the on-device loop over iterations
    std::vector<void*> rho;
    std::vector<const void*> V;
    bool begun = false;
    std::string err;
};

namespace {
dft_status bfail(dft_batch* b, dft_status code, const std::string& msg) {
    if (b) b->err = msg;
    else g_create_error = msg;
    return code;
}

void batch_release_graph(dft_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->loop = false;
}
}  // namespace

extern "C" {

dft_status dft_batch_create(const dft_params* params, int count, void* cuda_stream, dft_batch** out) {
    if (!params || !out || count < 1) return bfail(nullptr, DFT_EINVAL, "bad batch arguments");
    *out = nullptr;
    dft_batch* b = new dft_batch();
    if (cuda_stream) {
        b->main = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, DFT_ECUDA, "stream creation failed");
        }
        b->own_main = true;
    }
    cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < count; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            dft_batch_destroy(b);
            return bfail(nullptr, DFT_ECUDA, "stream creation failed");
        }
        b->streams.push_back(st);
        b->joins.push_back(ev);
        dft_plan* p = nullptr;
        dft_status s = dft_plan_create(&params[i], st, &p);
        if (s != DFT_OK) {
            const std::string msg = "state " + std::to_string(i) + ": " + g_create_error;
            dft_batch_destroy(b);
            return bfail(nullptr, s, msg);
        }
        b->plans.push_back(p);
    }
    *out = b;
    return DFT_OK;
}

dft_status dft_batch_destroy(dft_batch* b) {
    if (!b) return DFT_OK;
    batch_release_graph(b);
    for (dft_plan* p : b->plans) dft_plan_destroy(p);
    for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->joins) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_main) cudaStreamDestroy(b->main);
    delete b;
    return DFT_OK;
}

const char* dft_batch_last_error(const dft_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

dft_status dft_batch_begin(dft_batch* b, void* const* rho, const void* const* V) {
    if (!b || !rho || !V) return bfail(b, DFT_EINVAL, "NULL argument");
    batch_release_graph(b);
    b->rho.assign(rho, rho + b->plans.size());
    b->V.assign(V, V + b->plans.size());
    // all states start after work already queued on the main stream
    cudaEventRecord(b->fork, b->main);
    for (size_t i = 0; i < b->plans.size(); ++i) {
        cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        dft_status s = dft_iter_begin(b->plans[i], b->rho[i], b->V[i]);
        if (s != DFT_OK) return bfail(b, s, "state " + std::to_string(i) + ": " + b->plans[i]->err);
        cudaEventRecord(b->joins[i], b->streams[i]);
        cudaStreamWaitEvent(b->main, b->joins[i], 0);
    }
    b->begun = true;
    return DFT_OK;
}

dft_status dft_batch_autotune(dft_batch* b, void* const* rho, const void* const* V, int reps) {
    if (!b || !rho || !V) return bfail(b, DFT_EINVAL, "NULL argument");
    // each state's plan on its own fields, one state at a time (states of one grid share the
    // cached choice); the begun iteration and its graph no longer apply
    batch_release_graph(b);
    b->begun = false;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        dft_status s = dft_autotune(b->plans[i], rho[i], V[i], reps, nullptr);
        if (s != DFT_OK) return bfail(b, s, "state " + std::to_string(i) + ": " + b->plans[i]->err);
    }
    return DFT_OK;
}

dft_status dft_batch_iterate(dft_batch* b, int iters, double alpha_or_neg, double* resid_out) {
    if (!b || !b->begun) return bfail(b, DFT_EINVAL, "dft_batch_iterate needs a preceding dft_batch_begin");
    if (iters < 0) return bfail(b, DFT_EINVAL, "negative iteration count");
    if (b->exec && b->graph_alpha != alpha_or_neg) batch_release_graph(b);
    int* left = &b->plans[0]->ctl->loop_left;   // the loop's counter (in the first state's block)
    if (!b->exec) {
        // one iteration of every state: fork from the main stream, join back
        auto one_iteration = [&]() -> dft_status {
            cudaEventRecord(b->fork, b->main);
            dft_status st = DFT_OK;
            for (size_t i = 0; i < b->plans.size() && st == DFT_OK; ++i) {
                cudaStreamWaitEvent(b->streams[i], b->fork, 0);
                st = dft_iter_step(b->plans[i], b->rho[i], b->V[i], alpha_or_neg, nullptr, nullptr);
                if (st != DFT_OK) b->err = "state " + std::to_string(i) + ": " + b->plans[i]->err;
                cudaEventRecord(b->joins[i], b->streams[i]);
                cudaStreamWaitEvent(b->main, b->joins[i], 0);
            }
            return st;
        };
        // all iterations of all states in one graph launch (an on-device loop over the
        // captured iteration); a runtime without conditional graph nodes replays a graph of one
        cudaGraph_t g = nullptr;
        dft_status st = DFT_OK;
        cudaError_t e = build_loop_graph(b->main, left, &g, &st, one_iteration);
        if (e != cudaSuccess || st != DFT_OK) {
            // a runtime that does not capture programmatic edges: the states' passes in stream order
            bool any = false;
            for (dft_plan* q : b->plans) {
                any = any || q->g.pdl;
                q->g.pdl = 0;
                q->pdl_on = false;
            }
            if (any) {
                st = DFT_OK;
                e = build_loop_graph(b->main, left, &g, &st, one_iteration);
            }
        }
        if (st != DFT_OK) return st;
        b->loop = e == cudaSuccess;
        if (!b->loop) {
            e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return bfail(b, DFT_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
            st = one_iteration();
            e = cudaStreamEndCapture(b->main, &g);
            if (st != DFT_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return bfail(b, DFT_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
        }
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            batch_release_graph(b);
            return bfail(b, DFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        b->graph_alpha = alpha_or_neg;
    }
    if (b->loop && iters > 0) {
        k_loop_set<<<1, 1, 0, b->main>>>(left, iters);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->main);
        if (e != cudaSuccess) return bfail(b, DFT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    } else {
        for (int it = 0; it < iters; ++it) {
            cudaError_t e = cudaGraphLaunch(b->exec, b->main);
            if (e != cudaSuccess) return bfail(b, DFT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        }
    }
    if (resid_out) {
        cudaError_t e = cudaStreamSynchronize(b->main);
        if (e != cudaSuccess) return bfail(b, DFT_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
        for (size_t i = 0; i < b->plans.size(); ++i) {
            dft_status s = read_ctl(b->plans[i]);
            if (s != DFT_OK) return bfail(b, s, "state " + std::to_string(i) + ": " + b->plans[i]->err);
            resid_out[i] = b->plans[i]->ctl_host->resid;
        }
    }
    return DFT_OK;
}

dft_status dft_set_dependent_launch(dft_plan* p, int enable) {
    TRY(check_plan(p));
    // a captured iteration holds the launch attributes it was captured with
    release_iter_graph(p);
    p->pdl_on = enable != 0;
    p->g.pdl = (p->pdl_on && !p->prof) ? 1 : 0;
    describe_tuning(p);
    return DFT_OK;
}

dft_status dft_set_wait_polls(dft_plan* p, long long polls) {
    TRY(check_plan(p));
    if (polls < 0) return fail(p, DFT_EINVAL, "polls must be >= 0");
    // a captured iteration holds the old bound in its kernel parameters
    release_iter_graph(p);
    p->wait_polls = polls;
    return DFT_OK;
}

const char* dft_plan_tuning(const dft_plan* p) { return p ? p->tuning.c_str() : ""; }

dft_status dft_set_variants(dft_plan* p, int x_variant, int x_persistent, int y_variant, int z_variant) {
    TRY(check_plan(p));
    if (x_persistent < 0 || x_persistent > 2) return fail(p, DFT_EINVAL, "x_persistent is 0, 1 or 2");
    const std::vector<AxisPlan> orders = radix_orders(p->g.nx);
    if (x_variant < 0 || x_variant > (int)orders.size() || (x_variant == 0 && !dft_is_ct_size(p->g.nx)))
        return fail(p, DFT_EINVAL, "x variant out of range for this length");
    if (y_variant < 0 || y_variant > 1 || z_variant < 0 || z_variant > 3)
        return fail(p, DFT_EINVAL, "the y variant is 0 or 1, the z variant 0 to 3");
    p->g.xrt = x_variant > 0 ? 1 : 0;
    p->g.xpers = x_persistent;
    if (x_variant > 0) p->ax = orders[x_variant - 1];
    else dft_radix_plan(p->g.nx, &p->ax);
    p->g.yrt = y_variant;
    p->g.zgrp = z_variant & 1;
    p->g.zsplit = (z_variant >> 1) & 1;
    p->iter_ready = false;
    release_iter_graph(p);
    describe_tuning(p);
    return DFT_OK;
}

dft_status dft_profile_enable(dft_plan* p, int enable) {
    TRY(check_plan(p));
    collect_profile(p);
    for (int k = 0; k < K_COUNT; ++k) {
        p->prof_launches[k] = 0;
        p->prof_ms[k] = 0.0;
        p->prof_bytes[k] = 0.0;
    }
    p->prof = enable != 0;
    // per-pass event timing: each pass starts after the previous one has completed
    p->g.pdl = (p->pdl_on && !p->prof) ? 1 : 0;
    // the events of a full record batch created now, so that queuing profiled passes does not
    // wait on event creation (a slow host would otherwise leave gaps between the passes, which
    // the events around the next pass would count)
    if (p->prof) {
        const size_t need = 2 * (kProfBatch + 1);
        while (p->evpool.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return fail(p, DFT_ECUDA, "cudaEventCreate");
            p->evpool.push_back(e);
        }
    }
    return DFT_OK;
}

dft_status dft_profile_read(dft_plan* p, const char* name, int* launches, double* total_ms, double* total_bytes) {
    TRY(check_plan(p));
    if (!name) return fail(p, DFT_EINVAL, "NULL name");
    collect_profile(p);
    for (int k = 0; k < K_COUNT; ++k) {
        if (std::strcmp(name, kKindNames[k]) == 0) {
            if (launches) *launches = p->prof_launches[k];
            if (total_ms) *total_ms = p->prof_ms[k];
            if (total_bytes) *total_bytes = p->prof_bytes[k];
            return DFT_OK;
        }
    }
    return fail(p, DFT_EINVAL, std::string("unknown kernel name ") + name);
}

}  // extern "C"
