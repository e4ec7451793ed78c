// Shared-memory Stockham FFT of many independent lines.
//
// A CTA holds `lines` transforms of length n in shared memory; element e of
// line l sits at buf[e * es + l * ls].  Tiles of columns of the y / z axes use
// es = T (tile width), ls = 1 so that consecutive threads touch consecutive
// addresses; rows of the x axis use es = 1, ls = n + 1 (odd line pitch, free
// of bank conflicts for 8-byte elements).
//
// Stage with radix R and Ns = product of the earlier radices (self-sorting,
// out of place):  for butterfly j of n/R,
//     v[r] = src[j + r n/R] * w^( (j mod Ns) r n/(Ns R) ),  w = exp(-+2 pi i / n)
//     v    = DFT_R(v)
//     dst[(j / Ns) Ns R + (j mod Ns) + r Ns] = v[r]
// After all stages the result is in natural order.  The twiddle table holds
// exp(-2 pi i m / n), m < n, computed in double on the host.
#pragma once

#include "common.cuh"

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

// rotate by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot(C a) { return INV ? cmul_i(a) : cmul_mi(a); }

template <bool INV, typename C> __device__ __forceinline__ void dft3(C* v) {
    using R = decltype(C().x);
    const R h = R(0.86602540378443864676);   // sqrt(3)/2
    C s = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m = csub(v[0], cscale(s, R(0.5)));
    C t = rot<INV>(cscale(d, h));              // -i h d (forward)
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C a0 = cadd(x0, x2), a1 = csub(x0, x2);
    C a2 = cadd(x1, x3), a3 = rot<INV>(csub(x1, x3));
    x0 = cadd(a0, a2);
    x2 = csub(a0, a2);
    x1 = cadd(a1, a3);
    x3 = csub(a1, a3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* v) {
    using R = decltype(C().x);
    const R s = R(0.70710678118654752440);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    // o_k *= W8^k, W8 = exp(-+ 2 pi i / 8)
    o1 = INV ? cmake<C>((o1.x - o1.y) * s, (o1.x + o1.y) * s) : cmake<C>((o1.x + o1.y) * s, (o1.y - o1.x) * s);
    o2 = rot<INV>(o2);
    o3 = INV ? cmake<C>((-o3.x - o3.y) * s, (o3.x - o3.y) * s) : cmake<C>((o3.y - o3.x) * s, (-o3.x - o3.y) * s);
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft16(C* v) {
    using R = decltype(C().x);
    // Y_r = DFT4(v[r], v[r+4], v[r+8], v[r+12]);  X[k1 + 4 k2] = DFT4_r(W16^(r k1) Y_r[k1])
    C y[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        C a = v[r], b = v[r + 4], c = v[r + 8], d = v[r + 12];
        dft4<INV>(a, b, c, d);
        y[r * 4 + 0] = a; y[r * 4 + 1] = b; y[r * 4 + 2] = c; y[r * 4 + 3] = d;
    }
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), c2 = R(0.70710678118654752440);
    const R sg = INV ? R(1) : R(-1);
    // W16^m for m = r k1 in {0..9}: (cos(2 pi m/16), sg sin(2 pi m/16))
    const R wc[10] = {R(1), c1, c2, s1, R(0), -s1, -c2, -c1, R(-1), -c1};
    const R ws[10] = {R(0), s1, c2, c1, R(1), c1, c2, s1, R(0), -s1};
#pragma unroll
    for (int r = 1; r < 4; ++r) {
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            const int m = r * k1;
            y[r * 4 + k1] = cmul(y[r * 4 + k1], cmake<C>(wc[m], sg * ws[m]));
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C a = y[0 * 4 + k1], b = y[1 * 4 + k1], c = y[2 * 4 + k1], d = y[3 * 4 + k1];
        dft4<INV>(a, b, c, d);
        v[k1] = a; v[k1 + 4] = b; v[k1 + 8] = c; v[k1 + 12] = d;
    }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft_small(C* v) {
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else if constexpr (R == 8) dft8<INV>(v);
    else dft16<INV>(v);
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int n, int ns,
                                               int lines, int es, int ls, const C* __restrict__ tw) {
    const int m = n / R;
    const int twstep = n / (ns * R);
    const int total = m * lines;
    for (int task = threadIdx.x; task < total; task += blockDim.x) {
        const int line = task % lines;
        const int j = task / lines;
        const int k = j % ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * m) * es + line * ls];
        if (ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[k * r * twstep];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R, INV>(v);
        const int base = (j / ns) * ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * ns) * es + line * ls] = v[r];
    }
}

// Stage of an odd prime radix R without a dedicated butterfly (5 <= R <= DFT_MAX_PRIME): the
// R-point DFT by its definition, out_q = sum_r v_r W_R^(r q), W_R = exp(-+2 pi i / R).  The stage
// twiddle of v_r and W_R^(r q) are both powers of exp(-+2 pi i / n), so each term takes one
// table entry, tw[(k r n/(Ns R) + (r q mod R) n/R) mod n].  R^2 terms per butterfly, one output
// per thread.
template <bool INV, typename C>
__device__ __forceinline__ void stockham_stage_odd(const C* __restrict__ src, C* __restrict__ dst, int n, int ns,
                                                   int R, int lines, int es, int ls, const C* __restrict__ tw) {
    const int m = n / R;
    const int twstep = n / (ns * R);
    const int total = m * lines * R;
    // one output q of one butterfly per task (R times the tasks of a butterfly per thread)
    for (int task = threadIdx.x; task < total; task += blockDim.x) {
        const int q = task % R;
        const int bt = task / R;
        const int line = bt % lines;
        const int j = bt / lines;
        const int k = j % ns;
        const int base = (j / ns) * ns * R + k;
        C acc = cmake<C>(0, 0);
        int rq = 0;   // r q mod R
        for (int r = 0; r < R; ++r) {
            int e = k * r * twstep + rq * m;
            if (e >= n) e -= n;
            C w = tw[e];
            if (INV) w.y = -w.y;
            acc = cadd(acc, cmul(src[(j + r * m) * es + line * ls], w));
            rq += q;
            if (rq >= R) rq -= R;
        }
        dst[(base + q * ns) * es + line * ls] = acc;
    }
}

// Transform all lines held in `a` (b is scratch of the same size).  The caller must
// __syncthreads() before the call (data in a visible).  Returns the buffer holding
// the result; all threads see it on return.
template <bool INV, typename C>
__device__ C* smem_fft(C* a, C* b, const AxisPlan& p, int lines, int es, int ls, const C* tw) {
    int ns = 1;
    for (int s = 0; s < p.nstages; ++s) {
        const int R = p.radix[s];
        switch (R) {
            case 2: stockham_stage<2, INV>(a, b, p.n, ns, lines, es, ls, tw); break;
            case 3: stockham_stage<3, INV>(a, b, p.n, ns, lines, es, ls, tw); break;
            case 4: stockham_stage<4, INV>(a, b, p.n, ns, lines, es, ls, tw); break;
            case 8: stockham_stage<8, INV>(a, b, p.n, ns, lines, es, ls, tw); break;
            case 16: stockham_stage<16, INV>(a, b, p.n, ns, lines, es, ls, tw); break;
            default: stockham_stage_odd<INV>(a, b, p.n, ns, R, lines, es, ls, tw); break;
        }
        __syncthreads();
        C* t = a; a = b; b = t;
        ns *= R;
    }
    return a;
}

// ------------------------------------------------------------------------------------
// Compile-time transforms.  The same Stockham stages with the length, the radix plan and
// (for column tiles) the tile width known at compile time, so that index arithmetic is by
// constants and every loop unrolls.  Radix plan of n: the factors 3 first, then 16s, then
// one of 2/4/8 -- the same order as the run-time AxisPlan.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int ct_radix_at(int n, int s) {
    int m = n, k = 0;
    while (m % 3 == 0) { if (k == s) return 3; m /= 3; ++k; }
    while (m >= 16 && m % 16 == 0) { if (k == s) return 16; m /= 16; ++k; }
    if (m > 1) { if (k == s) return m; ++k; }
    return 0;
}
__host__ __device__ constexpr int ct_nstages(int n) { int s = 0; while (ct_radix_at(n, s) != 0) ++s; return s; }
__host__ __device__ constexpr int ct_ns_at(int n, int s) { int p = 1; for (int i = 0; i < s; ++i) p *= ct_radix_at(n, i); return p; }

constexpr int kFftThreads = 256;

// Compile-time x passes keep element e of a row at position e + floor(e / 16): the first
// Stockham stage writes its outputs with a stride of R (16) elements across threads, which the
// pad turns into 17 so the eight-byte stores of a half-warp hit distinct banks.
__host__ __device__ constexpr int ct_xpad(int e) { return e + (e >> 4); }

// Row pitch (elements) of the compile-time x passes: at least the padded row length, and,
// when a stage has M < 16 butterflies per row (16/M rows in one half-warp), congruent to M
// modulo 16 so that those rows fall into disjoint bank groups.
__host__ __device__ constexpr int ct_row_pitch(int n) {
    int msmall = 0;
    for (int s = 0; s < ct_nstages(n); ++s) {
        const int m = n / ct_radix_at(n, s);
        if (m < 16) msmall = m;
    }
    const int len = ct_xpad(n - 1) + 1;
    if (msmall == 0) return len | 1;
    return len + (((msmall - len) % 16) + 16) % 16;
}

// One stage.  COLS: lines are tile columns (element e of line l at e*T + l, line index fastest
// across threads); otherwise lines are rows (element e of line l at e + l*ls, e fastest).
// Rows: the padded position ct_xpad(a + r s) of the r-th element a butterfly touches splits
// into a per-thread part and a compile-time part when s is a multiple of 16 (then (a + r s) >> 4
// = (a >> 4) + r s / 16), or when every a + r s stays inside one block of 16 positions past a
// multiple of 16 (loads: a < M, 16 % M == 0; stores: NS R == 16).  The butterfly then addresses
// its elements at one base pointer plus constants.
template <int M, int R> __host__ __device__ constexpr bool ct_split_loads() { return M % 16 == 0 || 16 % M == 0; }
template <int NS, int R> __host__ __device__ constexpr bool ct_split_stores() { return NS % 16 == 0 || NS * R == 16; }

template <int N, int R, int NS, bool INV, bool COLS, int T, typename C>
__device__ __forceinline__ void ct_stage(const C* __restrict__ src, C* __restrict__ dst, int lines, int ls,
                                         const C* __restrict__ tw) {
    constexpr int M = N / R;
    constexpr int TWSTEP = N / (NS * R);
    const int total = COLS ? M * T : M * lines;
    if constexpr (!COLS && ct_split_loads<M, R>() && ct_split_stores<NS, R>()) {
#pragma unroll 2
        for (int task = threadIdx.x; task < total; task += kFftThreads) {
            const int j = task % M, line = task / M;
            const int k = j % NS;
            // loads: element j + r M at pad(j) + r (M + M / 16) (M a multiple of 16), or at
            // j + pad(r M) (j < M <= 16, 16 % M == 0)
            const C* s0 = src + line * ls + (M % 16 == 0 ? ct_xpad(j) : j);
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s0[M % 16 == 0 ? r * (M + M / 16) : ct_xpad(r * M)];
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[k * r * TWSTEP];
                    if (INV) w.y = -w.y;
                    v[r] = cmul(v[r], w);
                }
            }
            dft_small<R, INV>(v);
            // stores: element b + r NS, b = (j / NS) NS R + k, at pad(b) + r (NS + NS / 16) (NS a
            // multiple of 16), or at b + b / 16 + r NS (NS R = 16: b a multiple of 16 plus k < NS)
            const int b = (j / NS) * (NS * R) + k;
            C* d0 = dst + line * ls + ct_xpad(b);
#pragma unroll
            for (int r = 0; r < R; ++r) d0[NS % 16 == 0 ? r * (NS + NS / 16) : r * NS] = v[r];
        }
        return;
    }
#pragma unroll 2
    for (int task = threadIdx.x; task < total; task += kFftThreads) {
        int line, j;
        if constexpr (COLS) { line = task % T; j = task / T; }
        else { j = task % M; line = task / M; }
        const int k = j % NS;
        const int off = COLS ? line : line * ls;
        constexpr int ES = COLS ? T : 1;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * M;
            v[r] = src[(COLS ? e * ES : ct_xpad(e)) + off];
        }
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[k * r * TWSTEP];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R, INV>(v);
        const int base = (j / NS) * (NS * R) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = base + r * NS;
            dst[(COLS ? e * ES : ct_xpad(e)) + off] = v[r];
        }
    }
}

template <int N, bool INV, bool COLS, int T, int S, typename C>
__device__ __forceinline__ void ct_stages(C*& a, C*& b, int lines, int ls, const C* tw) {
    if constexpr (S < ct_nstages(N)) {
        constexpr int R = ct_radix_at(N, S);
        constexpr int NS = ct_ns_at(N, S);
        ct_stage<N, R, NS, INV, COLS, T>(a, b, lines, ls, tw);
        __syncthreads();
        C* t = a; a = b; b = t;
        ct_stages<N, INV, COLS, T, S + 1>(a, b, lines, ls, tw);
    }
}

// Compile-time counterpart of smem_fft (same contract).  COLS with tile width T, or rows
// with `lines` rows of pitch ls.
template <int N, bool INV, bool COLS, int T, typename C>
__device__ __forceinline__ C* ct_fft(C* a, C* b, int lines, int ls, const C* tw) {
    ct_stages<N, INV, COLS, T, 0>(a, b, lines, ls, tw);
    return a;
}

// Length-generic front end: N > 0 uses the compile-time stages, N == 0 the run-time plan.
template <int N, bool INV, bool COLS, int T, typename C>
__device__ __forceinline__ C* any_fft(C* a, C* b, const AxisPlan& p, int lines, int es, int ls, const C* tw) {
    if constexpr (N > 0) return ct_fft<N, INV, COLS, T>(a, b, lines, ls, tw);
    else return smem_fft<INV>(a, b, p, lines, es, ls, tw);
}

// ------------------------------------------------------------------------------------
// Grouped column transforms: `groups` tiles of T columns x N rows, tile g at offset g * GSTR,
// transformed together so that every stage has groups * T * N / R butterflies for the CTA's
// NT threads.  Inside a tile, element e of column t sits at T * ct_xpad(e) + t (padded: the
// first stage's outputs, R rows apart across threads, then fall into distinct bank groups);
// SRC_DENSE / DST_DENSE make the first stage read, or the last stage write, the dense layout
// e * T + t of a TMA box instead.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int ct_gpos(int e, int T) { return T * ct_xpad(e); }
__host__ __device__ constexpr int ct_gtile(int n, int T) { return T * (ct_xpad(n - 1) + 1); }
// group stride: the padded tile rounded up to 128 bytes (TMA destinations are 128-byte aligned)
__host__ __device__ constexpr int ct_gstride(int n, int T, int csize) {
    return (ct_gtile(n, T) + 128 / csize - 1) / (128 / csize) * (128 / csize);
}

// FOLD (a first stage only): the inputs of groups 3 and 4 are taken as group g - i kf.x group
// fold_partner(g) -- the y derivatives of the back convolution added before a z transform, where
// the wave number k_y is one constant per tile (kf.x = 0 leaves the groups as they are).
__host__ __device__ constexpr int fold_partner(int g) { return g == 4 ? 7 : 8; }

template <bool FOLD, int T, bool SD, int GSTR, typename C>
__device__ __forceinline__ void fold_input(C& v, const C* __restrict__ src, int e, int g, int off, C kf) {
    if constexpr (FOLD) {
        if ((g == 3 || g == 4) && kf.x != decltype(kf.x)(0)) {
            const C u = src[(SD ? e * T : ct_gpos(e, T)) + off + (fold_partner(g) - g) * GSTR];
            v.x += kf.x * u.y;
            v.y -= kf.x * u.x;
        }
    }
}

template <int N, int R, int NS, bool INV, int T, int GSTR, bool SD, bool DD, int NT, bool FOLD = false, typename C>
__device__ __forceinline__ void ct_stage_grouped(const C* __restrict__ src, C* __restrict__ dst, int groups,
                                                 const C* __restrict__ tw, C kf = C{}) {
    constexpr int M = N / R;
    constexpr int TWSTEP = N / (NS * R);
    constexpr int PERG = M * T;
    static_assert(!FOLD || NS == 1, "the fold belongs to a first stage");
    const int total = PERG * groups;
    for (int task = threadIdx.x; task < total; task += NT) {
        const int g = task / PERG;
        const int rem = task - g * PERG;
        const int t = rem % T, j = rem / T;
        const int k = j % NS;
        const int off = g * GSTR + t;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * M;
            v[r] = src[(SD ? e * T : ct_gpos(e, T)) + off];
            fold_input<FOLD, T, SD, GSTR>(v[r], src, e, g, off, kf);
        }
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[k * r * TWSTEP];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R, INV>(v);
        const int base = (j / NS) * (NS * R) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = base + r * NS;
            dst[(DD ? e * T : ct_gpos(e, T)) + off] = v[r];
        }
    }
}

template <int N, bool INV, int T, int GSTR, bool SD, bool DD, int NT, int S, bool FOLD = false, typename C>
__device__ __forceinline__ void ct_stages_grouped(C*& a, C*& b, int groups, const C* tw, C kf = C{}) {
    if constexpr (S < ct_nstages(N)) {
        constexpr int R = ct_radix_at(N, S);
        constexpr int NS = ct_ns_at(N, S);
        constexpr bool last = (S + 1 == ct_nstages(N));
        ct_stage_grouped<N, R, NS, INV, T, GSTR, SD && S == 0, DD && last, NT, FOLD && S == 0>(a, b, groups, tw, kf);
        __syncthreads();
        C* t = a; a = b; b = t;
        ct_stages_grouped<N, INV, T, GSTR, SD, DD, NT, S + 1>(a, b, groups, tw);
    }
}

// Transform `groups` tiles held in a (b: scratch of the same size); the caller syncs before;
// returns the buffer holding the result (synced).  FOLD: see ct_stage_grouped (kf.x = k_y).
template <int N, bool INV, int T, int GSTR, bool SD = false, bool DD = false, int NT = kFftThreads,
          bool FOLD = false, typename C>
__device__ __forceinline__ C* ct_fft_grouped(C* a, C* b, int groups, const C* tw, C kf = C{}) {
    ct_stages_grouped<N, INV, T, GSTR, SD, DD, NT, 0, FOLD>(a, b, groups, tw, kf);
    return a;
}

// ------------------------------------------------------------------------------------
// In-place grouped column transforms (same layouts, SRC_DENSE / DST_DENSE meaning and twiddle
// table as ct_fft_grouped).  Each thread takes one butterfly of a stage, holds its R inputs in
// registers across a barrier and then writes its outputs over the same tile, so that no scratch
// tiles are needed; the groups are taken in chunks of NT / (T N / R) per pass of the threads
// (chunks touch disjoint groups, so one barrier per chunk orders its reads before its writes).
// The caller syncs before the call; the last stage is NOT followed by a barrier, so the caller
// syncs (after any proxy fence its TMA stores need) before reading the result.
// ------------------------------------------------------------------------------------
// barrier among the first `count` threads of the CTA (a multiple of 32), named barrier 1
__device__ __forceinline__ void bar_sync_first(int count) {
    asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}

template <int N, int R, int NS, bool INV, int T, int GSTR, bool SD, bool DD, int NT, bool END_SYNC, bool FOLD = false,
          typename C>
__device__ __forceinline__ void ct_stage_grouped_ip(C* buf, int groups, const C* __restrict__ tw, C kf = C{}) {
    constexpr int M = N / R;
    constexpr int TWSTEP = N / (NS * R);
    constexpr int PERG = M * T;
    static_assert(PERG <= NT, "the butterflies of one group fit the threads of a pass");
    constexpr int GCH = NT / PERG;
    // the thread index read through a volatile move: the compiler would otherwise hoist every
    // stage's butterfly offsets (loop invariants of a persistent kernel's tile loop) and keep
    // them all live across the loop
    int tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int gl = tid / PERG;
    const int rem = tid - gl * PERG;
    const int t = rem % T, j = rem / T;
    const int k = j % NS;
    const int base = (j / NS) * (NS * R) + k;
    for (int g0 = 0; g0 < groups; g0 += GCH) {
        const int ng = groups - g0 < GCH ? groups - g0 : GCH;
        // the warps that hold this chunk's butterflies take part (named barrier among them);
        // their idle lanes transform a copy of the chunk's first group and do not store it
        const int nthr = (ng * PERG + 31) & ~31;
        if (tid < nthr) {
            const bool act = gl < ng;
            const int g = g0 + (act ? gl : 0);
            const int off = g * GSTR + t;
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = j + r * M;
                v[r] = buf[(SD ? e * T : ct_gpos(e, T)) + off];
                // the fold's partner groups lie past the transformed ones: never written here
                fold_input<FOLD, T, SD, GSTR>(v[r], buf, e, g, off, kf);
            }
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[k * r * TWSTEP];
                    if (INV) w.y = -w.y;
                    v[r] = cmul(v[r], w);
                }
            }
            dft_small<R, INV>(v);
            bar_sync_first(nthr);
            if (act) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = base + r * NS;
                    buf[(DD ? e * T : ct_gpos(e, T)) + off] = v[r];
                }
            }
        }
    }
    if constexpr (END_SYNC) __syncthreads();
}

template <int N, bool INV, int T, int GSTR, bool SD, bool DD, int NT, int S, bool FOLD = false, typename C>
__device__ __forceinline__ void ct_stages_grouped_ip(C* a, int groups, const C* tw, C kf = C{}) {
    if constexpr (S < ct_nstages(N)) {
        constexpr int R = ct_radix_at(N, S);
        constexpr int NS = ct_ns_at(N, S);
        constexpr bool last = (S + 1 == ct_nstages(N));
        ct_stage_grouped_ip<N, R, NS, INV, T, GSTR, SD && S == 0, DD && last, NT, !last, FOLD && S == 0>(a, groups,
                                                                                                       tw, kf);
        ct_stages_grouped_ip<N, INV, T, GSTR, SD, DD, NT, S + 1>(a, groups, tw);
    }
}

// Transform `groups` tiles held in a, in place; the caller syncs before and after.  FOLD: see
// ct_stage_grouped (the partner groups must lie at or past `groups`).
template <int N, bool INV, int T, int GSTR, bool SD = false, bool DD = false, int NT = kFftThreads,
          bool FOLD = false, typename C>
__device__ __forceinline__ void ct_fft_grouped_ip(C* a, int groups, const C* tw, C kf = C{}) {
    ct_stages_grouped_ip<N, INV, T, GSTR, SD, DD, NT, 0, FOLD>(a, groups, tw, kf);
}
