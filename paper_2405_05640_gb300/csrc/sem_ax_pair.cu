// sem_ax_pair.cu -- the FP64 local stiffness operator w = A_L u evaluated in
// FP32-pair ("double-float") arithmetic.
//
// The operator is the one of sem_ax.cu (paper section 3.1: element by element,
// matrix free; u_r = D u along each direction, v = G (u_r, u_s, u_t) with the
// six symmetric geometric factors, w = D^T v_r + D^T v_s + D^T v_t).
//
// Why a second FP64 kernel: GB300 issues FP64 FMAs at 2 per clock per SM
// against 128 FP32 FMAs, and converts between FP32 and FP64 at the same slow
// rate (both measured).  A plain FP64 A_L needs ~57 FMAs per point and is
// bound by the FP64 pipe at about a tenth of HBM bandwidth.  Here every FP64
// value is carried as hi + lo (two floats, 48 significant bits) and the work
// runs on the FP32 pipes:
//  - FP64 -> pair: integer bit operations (truncated 24-bit hi, the remaining
//    29 mantissa bits rounded into lo), after scaling the element by a power
//    of two so that its largest value lies in [1, 2);
//  - a product a*b of pairs: p = fl(ah*bh), its exact error fma(ah, bh, -p),
//    and the cross terms ah*bl + al*bh;
//  - the sum along a line (the N+1 terms of one derivative): the running sum
//    starts at a power-of-two anchor sigma >= 2 sum |terms|, so |sum| >= |term|
//    always holds, s1 - s is exact (Fast2Sum) and the product's and the
//    addition's rounding errors together are one FMA, dh*xh - (s1 - s);
//    sigma is subtracted exactly at the end (Sterbenz);
//  - pair -> FP64: two conversions and one FP64 add per point (FP64 pipe,
//    parallel to the FP32 work), then the exponent shift undone on the bits.
// The error is about 2^-42 of the line-wise magnitudes |D^T||G||D||u| (FP64
// proper: ~2^-50); on fields without strong cancellation that is within
// 1e-12 of the FP64 result in the relative 2-norm.
//
// Layout per element (one CTA at a time, persistent grid): the G pair slab
// [6][npt] (48 bytes per point, contiguous) arrives by a 1-D bulk copy (TMA)
// on an mbarrier, u is prefetched into registers one element ahead (coalesced
// loads); the pair fields live in shared memory with an
// odd padded stride per r-line, so that lines of all three directions are
// read without bank conflicts.  2 threads per line (each half of the
// outputs), the halves warp-aligned so that D (in the kernel parameters,
// constant bank) is a uniform operand of every FMA.

#include <algorithm>
#include <cmath>

#include "sem_common.cuh"

namespace sem {

template <int N1>
struct PairD {
    float h[N1 * N1], l[N1 * N1];  // D = h + l, row-major D[i][l]
    float rf[N1], rb[N1];           // anchor factors: 2 sum_l |h[i][l]| and 2 sum_l |h[l][i]|, rounded up
    // the same entries for two consecutive outputs i, i+1 side by side (packed
    // FP32x2 operands): fh[i][l] = (h[i][l], h[i+1][l]), bh[i][l] = (h[l][i], h[l][i+1])
    float2 fh[(N1 - 1) * N1], fl[(N1 - 1) * N1], bh[(N1 - 1) * N1], bl[(N1 - 1) * N1];
};

struct PairArgs {
    int64_t E;
    int nst;             // pipeline stages of the G slab (1..2)
    int use_tma;         // bulk-copy staging of G (else plain loads)
};

template <int N>
struct PairShape {
    static constexpr int N1 = N + 1;
    static constexpr int NPT = N1 * N1 * N1;
    static constexpr int NL = N1 * N1;                      // lines per direction
    static constexpr int S = (N1 % 2 == 0) ? N1 + 1 : N1;   // odd pair stride of an r-line
    static constexpr int LP = (NL + 31) / 32 * 32;          // threads per half (warp multiple)
    static constexpr int T = 2 * LP;                        // threads per CTA
    static constexpr int H0 = (N1 + 1) / 2;                 // half 0: outputs [0, H0)
    static constexpr int PB = S * NL;                       // pairs in one padded field
    static constexpr int UPT = (NPT + T - 1) / T;           // u values per thread (prefetched)
    static constexpr int SB = NPT * 48;                     // one stage: the G pair slab
    // stages, 4 pair fields, 8 mbarriers, 16 ints and 16 doubles of reductions
    static constexpr int smem(int nst) { return nst * SB + 4 * PB * 8 + 64 + 16 * 4 + 16 * 8; }
};

// ---------------------------------------------------------------- pair arithmetic

// FP64 -> pair, with the element exponent shift sc (value * 2^-sc).
__device__ __forceinline__ float2 split_f64(double u, int sc) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sgn = hw & 0x80000000u;
    const int ex = (int)((hw >> 20) & 0x7ffu) - sc;  // scaled biased exponent (<= 1023)
    const int eh = ex - 896;                          // float exponent field of hi
    const int el = ex - 948;                          // float exponent field of 2^(ex-1075)
    const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned hb = sgn | ((unsigned)eh << 23) | m23;
    const float hi = __uint_as_float(eh >= 1 ? hb : sgn);
    const float lmag = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)(el > 0 ? el : 1) << 23));
    const float lo = __uint_as_float(el >= 1 ? (__float_as_uint(lmag) | sgn) : 0u);
    return make_float2(hi, lo);
}

// pair -> FP64, undoing the exponent shift sc.
__device__ __forceinline__ double pair_to_f64(float2 v, int sc) {
    const double r = __dadd_rn((double)v.x, (double)v.y);
    long long b = __double_as_longlong(r);
    const int ex = (int)((b >> 52) & 0x7ff);
    const int ne = ex + sc;
    if (ex == 0 || ne <= 0) return 0.0;
    b += (long long)sc << 52;
    return __longlong_as_double(b);
}

// (hi, lo) -> (hi + lo, rest) by Fast2Sum (three additions).  Exact when
// |hi| >= |lo|; when |lo| > |hi| (a value that cancelled to a few units of
// its anchor) the error stays a few units of 2^-24 of that tiny value.  Keeps
// low parts small, so that their FP32 products stay at the format's accuracy.
__device__ __forceinline__ float2 pair_fast(float hi, float lo) {
    const float q = __fadd_rn(hi, lo);
    return make_float2(q, __fsub_rn(lo, __fsub_rn(q, hi)));
}

// a + b: TwoSum of the high parts, low parts added.  Used only where the
// result is added again or converted to FP64, never multiplied, so it is not
// renormalised.
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bv = __fsub_rn(s, a.x);
    const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bv)), __fsub_rn(b.x, bv));
    return make_float2(s, __fadd_rn(__fadd_rn(t, a.y), b.y));
}

// g0 x0 + g1 x1 + g2 x2 for pairs (the geometric-factor products of one point).
__device__ __forceinline__ float2 pair_dot3(float2 g0, float2 x0, float2 g1, float2 x1, float2 g2, float2 x2) {
    const float p0 = __fmul_rn(g0.x, x0.x), p1 = __fmul_rn(g1.x, x1.x), p2 = __fmul_rn(g2.x, x2.x);
    float c = __fadd_rn(__fadd_rn(fmaf(g0.x, x0.x, -p0), fmaf(g1.x, x1.x, -p1)), fmaf(g2.x, x2.x, -p2));
    c = fmaf(g0.x, x0.y, c);
    c = fmaf(g0.y, x0.x, c);
    c = fmaf(g1.x, x1.y, c);
    c = fmaf(g1.y, x1.x, c);
    c = fmaf(g2.x, x2.y, c);
    c = fmaf(g2.y, x2.x, c);
    // TwoSum(p0, p1), TwoSum(s, p2)
    float s = __fadd_rn(p0, p1);
    float bv = __fsub_rn(s, p0);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(p0, __fsub_rn(s, bv)), __fsub_rn(p1, bv)));
    const float s2 = __fadd_rn(s, p2);
    bv = __fsub_rn(s2, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bv)), __fsub_rn(p2, bv)));
    return pair_fast(s2, c);
}

// One line of a derivative contraction, outputs [I0, I1):
//   y_i = sum_l Dm(i, l) x_l,  Dm = D (TR = false) or D^T (TR = true).
// Anchor of output i: sigma_i = the power of two >= rf_i max_l |x_l.hi|
// (rf_i >= 2 sum_l |Dm(i,l)|), so sigma_i >= 2 sum_l |p_l| and the running
// sum stays in [sigma_i / 2, 3 sigma_i / 2]: s1 - s is exact (Fast2Sum) and
// the whole error of adding the exact product, dh*xh - (s1 - s), is formed by
// one FMA.  Seven FP32 instructions per term; two error accumulators (sum
// errors; cross terms) keep the dependency chains short.  Forward outputs
// (multiplied by G next) are renormalised, backward ones (only added) not.
template <int N1, int I0, int I1, bool TR>
__device__ __forceinline__ void line_dot(const float2 (&x)[N1], const PairD<N1> &D, float2 *y) {
    float m = 0.f;
#pragma unroll
    for (int l = 0; l < N1; ++l) m = fmaxf(m, fabsf(x[l].x));
    // outputs in pairs (i, i+1): every FP32 operation below runs as one packed
    // FP32x2 instruction for both (the same IEEE operations per lane as the
    // scalar tail; -(s1 - s) is fma(s1, -1, s), exact)
    constexpr int NP = (I1 - I0) / 2;
    if constexpr (NP > 0) {
        float2 xh[N1], xl[N1];
#pragma unroll
        for (int l = 0; l < N1; ++l) {
            xh[l] = make_float2(x[l].x, x[l].x);
            xl[l] = make_float2(x[l].y, x[l].y);
        }
        const float2 minus1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            const int i = I0 + 2 * pr;
            float2 sig;
            {
                const float f0 = __fmul_rn(m, TR ? D.rb[i] : D.rf[i]);
                const float f1 = __fmul_rn(m, TR ? D.rb[i + 1] : D.rf[i + 1]);
                sig = make_float2(__int_as_float((__float_as_int(f0) + 0x007fffff) & 0x7f800000),
                                  __int_as_float((__float_as_int(f1) + 0x007fffff) & 0x7f800000));
            }
            float2 s2 = sig, ce = make_float2(0.f, 0.f), cx = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < N1; ++l) {
                const float2 dh = TR ? D.bh[i * N1 + l] : D.fh[i * N1 + l];
                const float2 dl = TR ? D.bl[i * N1 + l] : D.fl[i * N1 + l];
                const float2 p = __fmul2_rn(dh, xh[l]);
                const float2 s1 = __fadd2_rn(s2, p);
                const float2 nd = __ffma2_rn(s1, minus1, s2);  // s - s1, exact: |s| >= |p|
                ce = __fadd2_rn(ce, __ffma2_rn(dh, xh[l], nd)); // fl(dh*xh - (s1 - s))
                s2 = s1;
                cx = __ffma2_rn(dh, xl[l], cx);
                cx = __ffma2_rn(dl, xh[l], cx);
            }
            const float2 hi = __fadd2_rn(s2, make_float2(-sig.x, -sig.y));  // exact (Sterbenz)
            const float2 lo = __fadd2_rn(ce, cx);
            y[i - I0] = TR ? make_float2(hi.x, lo.x) : pair_fast(hi.x, lo.x);
            y[i + 1 - I0] = TR ? make_float2(hi.y, lo.y) : pair_fast(hi.y, lo.y);
        }
    }
#pragma unroll
    for (int i = I0 + 2 * NP; i < I1; ++i) {  // the odd output, scalar
        const float f = __fmul_rn(m, TR ? D.rb[i] : D.rf[i]);
        const float sig = __int_as_float((__float_as_int(f) + 0x007fffff) & 0x7f800000);
        float s = sig, ce = 0.f, cx = 0.f;
#pragma unroll
        for (int l = 0; l < N1; ++l) {
            const float dh = TR ? D.h[l * N1 + i] : D.h[i * N1 + l];
            const float dl = TR ? D.l[l * N1 + i] : D.l[i * N1 + l];
            const float p = __fmul_rn(dh, x[l].x);
            const float s1 = __fadd_rn(s, p);
            const float d = __fsub_rn(s1, s);                 // exact: |s| >= |p|
            ce = __fadd_rn(ce, fmaf(dh, x[l].x, -d));          // = fl(dh*xh - (s1 - s))
            s = s1;
            cx = fmaf(dh, x[l].y, cx);
            cx = fmaf(dl, x[l].x, cx);
        }
        const float hi = __fsub_rn(s, sig), lo = __fadd_rn(ce, cx);  // s - sigma exact (Sterbenz)
        y[i - I0] = TR ? make_float2(hi, lo) : pair_fast(hi, lo);
    }
}

// Line geometry: points of line L of direction dir (0 r, 1 s, 2 t) in the
// padded pair layout are base + l * step.
template <int N>
__device__ __forceinline__ void line_at(int dir, int L, int &base, int &step) {
    using P = PairShape<N>;
    constexpr int N1 = P::N1, S = P::S;
    if (dir == 0) {  // (., j, k), L = j + N1 k
        base = S * L;
        step = 1;
    } else if (dir == 1) {  // (i, ., k), L = i + N1 k
        base = S * N1 * (L / N1) + L % N1;
        step = S;
    } else {  // (i, j, .), L = i + N1 j
        base = S * (L / N1) + L % N1;
        step = S * N1;
    }
}

template <int N>
__device__ __forceinline__ int padded(int p) {
    using P = PairShape<N>;
    return P::S * (p / P::N1) + p % P::N1;
}

// Forward contraction of one line into dst (outputs of half H).
template <int N, int H>
__device__ __forceinline__ void fwd_line(const float2 *src, float2 *dst, int base, int step, const PairD<N + 1> &D) {
    using P = PairShape<N>;
    constexpr int N1 = P::N1, I0 = H ? P::H0 : 0, I1 = H ? N1 : P::H0;
    float2 x[N1], y[I1 - I0];
#pragma unroll
    for (int l = 0; l < N1; ++l) x[l] = src[base + l * step];
    line_dot<N1, I0, I1, false>(x, D, y);
#pragma unroll
    for (int i = I0; i < I1; ++i) dst[base + i * step] = y[i - I0];
}

// Backward contraction of one line; mode 0: write into acc, 1: add into acc,
// 2: add acc and store the FP64 result (scaled back by sc) to global; with pe
// (fused CG form) also pw += pe * w at the stored points.
template <int N, int H, int MODE>
__device__ __forceinline__ void bwd_line(const float2 *src, float2 *acc, int base, int step, const PairD<N + 1> &D,
                                         double *__restrict__ we, int gbase, int gstep, int sc, bool nan,
                                         const double *pe = nullptr, double *pw = nullptr) {
    using P = PairShape<N>;
    constexpr int N1 = P::N1, I0 = H ? P::H0 : 0, I1 = H ? N1 : P::H0;
    float2 x[N1], y[I1 - I0];
#pragma unroll
    for (int l = 0; l < N1; ++l) x[l] = src[base + l * step];
    line_dot<N1, I0, I1, true>(x, D, y);
#pragma unroll
    for (int i = I0; i < I1; ++i) {
        const int q = base + i * step;
        if (MODE == 0) {
            acc[q] = y[i - I0];
        } else if (MODE == 1) {
            acc[q] = pair_add(acc[q], y[i - I0]);
        } else {
            const float2 v = pair_add(acc[q], y[i - I0]);
            const double wv = nan ? __longlong_as_double(0x7ff8000000000000ll) : pair_to_f64(v, sc);
            we[gbase + i * gstep] = wv;
            if (pe) *pw = fma(pe[gbase + i * gstep], wv, *pw);
        }
    }
}

// CG: the fused CG form of the FP64 solver: p <- dinv r + beta p (FP64,
// written back), w = A_L p, and sum_l p_l w_l reduced over the grid into
// alpha = rho / pw (per-CTA partials; the last CTA sums them in a fixed order).
template <int N, bool CG>
__global__ void __launch_bounds__(PairShape<N>::T)
    ax_pair_kernel(const double *__restrict__ u, double *__restrict__ w, const float2 *__restrict__ G2,
                   const PairD<N + 1> D, const PairArgs a, const CgFuse<double> cg, int *__restrict__ err) {
    using P = PairShape<N>;
    constexpr int N1 = P::N1, NPT = P::NPT, NL = P::NL, LP = P::LP, T = P::T, PB = P::PB;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nst = a.nst;
    float2 *U = reinterpret_cast<float2 *>(smem + nst * P::SB);  // u pairs, later W
    float2 *R = U + PB, *Sb = R + PB, *Tb = Sb + PB;             // u_r, u_s, u_t, later v_*
    uint64_t *bar = reinterpret_cast<uint64_t *>(Tb + PB);
    int *red = reinterpret_cast<int *>(bar + 8);
    double *dred = reinterpret_cast<double *>(red + 16);
    if (CG && cg.scal->done) return;  // uniform: the solve has converged
    const int tid = threadIdx.x;
    const int half = tid / LP, L = tid % LP;  // warp-uniform half
    const bool lact = L < NL;
    const int lane = tid & 31, wid = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t E = a.E, stride = gridDim.x;
    auto issue = [&](int64_t e, int s) {
        mbar_arrive_expect_tx(&bar[s], P::SB);
        bulk_g2s(smem + s * P::SB, G2 + e * 6 * NPT, P::SB, &bar[s]);
    };
    if (a.use_tma && tid == 0)
        for (int s = 0; s < nst; ++s) {
            const int64_t e = blockIdx.x + s * stride;
            if (e < E) issue(e, s);
        }
    // the operand of the element being processed (u; CG: r, dinv and the old
    // p), prefetched into registers one element ahead.  In the CG form p of a
    // later element is still the old one when prefetched: this CTA writes it
    // only when it reaches that element.
    double ur[P::UPT], rr[CG ? P::UPT : 1], dr[CG ? P::UPT : 1];
    const double beta = CG ? cg.scal->beta : 0.0;
    double pw_acc = 0.0;
    auto load_u = [&](int64_t e) {
#pragma unroll
        for (int q = 0; q < P::UPT; ++q) {
            const int idx = tid + q * T;
            const bool in = e < E && idx < NPT;
            if (CG) {
                ur[q] = in ? cg.p[e * NPT + idx] : 0.0;
                rr[q] = in ? __ldg(cg.r + e * NPT + idx) : 0.0;
                dr[q] = in ? __ldg(cg.dinv + e * NPT + idx) : 0.0;
            } else {
                ur[q] = in ? __ldg(u + e * NPT + idx) : 0.0;
            }
        }
    };
    load_u(blockIdx.x);

    int it = 0;
    bool ok = true;
    for (int64_t e = blockIdx.x; e < E; e += stride, ++it) {
        const int s = it % nst;
        const float2 *sg = reinterpret_cast<const float2 *>(smem + s * P::SB);
        if (a.use_tma) {
            const bool mine = mbar_wait_bounded(&bar[s], (it / nst) & 1, err, kDevTimeoutTma);
            ok = __syncthreads_and(mine);
            if (!ok) break;
        } else {
            __syncthreads();
            float2 *dg = reinterpret_cast<float2 *>(smem + s * P::SB);
            for (int q = tid; q < 6 * NPT; q += T) dg[q] = G2[e * 6 * NPT + q];
            __syncthreads();
        }
        if (CG) {
            // p <- dinv r + beta p, the new search direction (FP64)
#pragma unroll
            for (int q = 0; q < P::UPT; ++q) {
                const int idx = tid + q * T;
                ur[q] = fma(beta, ur[q], dr[q] * rr[q]);
                if (idx < NPT) cg.p[e * NPT + idx] = ur[q];
            }
        }
        // element exponent: the largest biased FP64 exponent of u
        int exm = 0;
#pragma unroll
        for (int q = 0; q < P::UPT; ++q) exm = max(exm, (int)((__double_as_longlong(ur[q]) >> 52) & 0x7ff));
        exm = __reduce_max_sync(0xffffffffu, exm);
        if (lane == 0) red[wid] = exm;
        __syncthreads();
        exm = 0;
#pragma unroll
        for (int q = 0; q < T / 32; ++q) exm = max(exm, red[q]);
        const bool nan = exm == 0x7ff;
        const int sc = exm == 0 ? 0 : exm - 1023;
#pragma unroll
        for (int q = 0; q < P::UPT; ++q) {
            const int idx = tid + q * T;
            if (idx < NPT) U[padded<N>(idx)] = split_f64(ur[q], sc);
        }
        load_u(e + stride);  // in flight during the contractions
        __syncthreads();
        // u_r, u_s, u_t
        if (lact) {
            int base, step;
#pragma unroll
            for (int dir = 0; dir < 3; ++dir) {
                float2 *dst = dir == 0 ? R : (dir == 1 ? Sb : Tb);
                line_at<N>(dir, L, base, step);
                if (half == 0)
                    fwd_line<N, 0>(U, dst, base, step, D);
                else
                    fwd_line<N, 1>(U, dst, base, step, D);
            }
        }
        __syncthreads();
        // v = G (u_r, u_s, u_t), in place
        for (int q = tid; q < NPT; q += T) {
            const int pq = padded<N>(q);
            const float2 xr = R[pq], xs = Sb[pq], xt = Tb[pq];
            const float2 g0 = sg[q], g1 = sg[NPT + q], g2 = sg[2 * NPT + q];
            const float2 g3 = sg[3 * NPT + q], g4 = sg[4 * NPT + q], g5 = sg[5 * NPT + q];
            R[pq] = pair_dot3(g0, xr, g3, xs, g4, xt);
            Sb[pq] = pair_dot3(g3, xr, g1, xs, g5, xt);
            Tb[pq] = pair_dot3(g4, xr, g5, xs, g2, xt);
        }
        __syncthreads();  // stage s consumed: refill it while the backward pass runs
        if (a.use_tma && tid == 0) {
            const int64_t en = e + nst * stride;
            if (en < E) {
                fence_proxy_async_smem();
                issue(en, s);
            }
        }
        // w = D^T v_r + D^T v_s + D^T v_t, accumulated in U
        double *we = w + e * NPT;
        if (lact) {
            int base, step;
            line_at<N>(0, L, base, step);
            if (half == 0)
                bwd_line<N, 0, 0>(R, U, base, step, D, we, 0, 0, sc, nan);
            else
                bwd_line<N, 1, 0>(R, U, base, step, D, we, 0, 0, sc, nan);
        }
        __syncthreads();
        if (lact) {
            int base, step;
            line_at<N>(1, L, base, step);
            if (half == 0)
                bwd_line<N, 0, 1>(Sb, U, base, step, D, we, 0, 0, sc, nan);
            else
                bwd_line<N, 1, 1>(Sb, U, base, step, D, we, 0, 0, sc, nan);
        }
        __syncthreads();
        if (lact) {
            int base, step;
            line_at<N>(2, L, base, step);
            const int gbase = L, gstep = NL;  // (i, j, k): i + N1 j + N1^2 k, L = i + N1 j
            const double *pe = CG ? cg.p + e * NPT : nullptr;  // written above, visible after the barriers
            if (half == 0)
                bwd_line<N, 0, 2>(Tb, U, base, step, D, we, gbase, gstep, sc, nan, pe, &pw_acc);
            else
                bwd_line<N, 1, 2>(Tb, U, base, step, D, we, gbase, gstep, sc, nan, pe, &pw_acc);
        }
        // the barrier at the top of the next element protects U, R, Sb, Tb
    }
    if (!ok && a.use_tma && tid == 0) {
        // a wait gave up: drain the copies this CTA still has in flight (bounded)
        for (int s = 0; s < nst; ++s) {
            const int itn = it + ((s - it % nst) + nst) % nst;
            const int64_t en = blockIdx.x + (int64_t)itn * stride;
            if (en < E) mbar_wait_bounded(&bar[s], (itn / nst) & 1, err, kDevTimeoutTma);
        }
    }
    if (CG) {
        // grid reduction of p.w: per-CTA partials, the last CTA sums them with
        // all its threads in a fixed order
        __shared__ int s_last;
        double v = pw_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) dred[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < T / 32; ++q) t += dred[q];
            cg.partial[blockIdx.x] = t;
            __threadfence();
            s_last = atomicAdd(&cg.scal->cnt[3], 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double t = 0.0;
            for (int q = tid; q < (int)gridDim.x; q += T) t += __ldcg(cg.partial + q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) dred[wid] = t;  // thread 0 read dred before the barrier above
            __syncthreads();
            if (tid == 0) {
                double pw = 0.0;
                for (int q = 0; q < T / 32; ++q) pw += dred[q];
                cg.scal->pw = pw;
                cg.scal->alpha = cg.scal->rho / pw;
                cg.scal->cnt[3] = 0u;
            }
        }
    }
}

// ---------------------------------------------------------------- launch

AxTune g_ax_pair_tune[kMaxN1] = {};

template <int N, bool CG>
static int launch_pair_n(const sem_mesh *m, const double *u, double *w, const CgFuse<double> &cg, cudaStream_t st) {
    using P = PairShape<N>;
    constexpr int N1 = P::N1;
    PairD<N1> D;
    for (int i = 0; i < N1; ++i)
        for (int l = 0; l < N1; ++l) {
            const double d = m->D.d[i * N1 + l];
            const float h = (float)d;
            D.h[i * N1 + l] = h;
            D.l[i * N1 + l] = (float)(d - (double)h);
        }
    for (int i = 0; i + 1 < N1; ++i)
        for (int l = 0; l < N1; ++l) {
            D.fh[i * N1 + l] = make_float2(D.h[i * N1 + l], D.h[(i + 1) * N1 + l]);
            D.fl[i * N1 + l] = make_float2(D.l[i * N1 + l], D.l[(i + 1) * N1 + l]);
            D.bh[i * N1 + l] = make_float2(D.h[l * N1 + i], D.h[l * N1 + i + 1]);
            D.bl[i * N1 + l] = make_float2(D.l[l * N1 + i], D.l[l * N1 + i + 1]);
        }
    for (int i = 0; i < N1; ++i) {
        double rs = 0.0, cs = 0.0;
        for (int l = 0; l < N1; ++l) {
            rs += std::fabs((double)D.h[i * N1 + l]);
            cs += std::fabs((double)D.h[l * N1 + i]);
        }
        // 2 x the absolute row (column) sum, enlarged by 2^-20 to cover the
        // rounding of the products and of m * rf in the kernel
        D.rf[i] = (float)(2.0 * rs * (1.0 + std::ldexp(1.0, -20)));
        D.rb[i] = (float)(2.0 * cs * (1.0 + std::ldexp(1.0, -20)));
    }
    AxTune tune = g_ax_pair_tune[N];
    int nst = tune.nst < 1 ? 1 : (tune.nst > 2 ? 2 : tune.nst);
    int dev_max = 0;
    SEM_CUDA_CHECK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    while (nst > 1 && P::smem(nst) > dev_max) --nst;
    const int smem = P::smem(nst);
    if (smem > dev_max) return fail(SEM_ERR_UNSUPPORTED, "element does not fit in shared memory");
    auto kern = ax_pair_kernel<N, CG>;
    SEM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P::T, smem));
    if (per_sm < 1) per_sm = 1;
    if (tune.per_sm_cap > 0 && per_sm > tune.per_sm_cap) per_sm = tune.per_sm_cap;
    int64_t grid = (int64_t)m->num_sms * per_sm;
    if (grid > m->E) grid = m->E;
    if (grid > kAxMaxGrid) grid = kAxMaxGrid;  // partials of the fused CG form
    PairArgs a;
    a.E = m->E;
    a.nst = nst;
    a.use_tma = reinterpret_cast<uintptr_t>(m->G2) % 16 == 0;
    kern<<<(int)grid, P::T, smem, st>>>(u, w, m->G2, D, a, cg, m->d_err);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

template <bool CG>
static int dispatch_pair(const sem_mesh *m, const double *u, double *w, const CgFuse<double> &cg, cudaStream_t st) {
    if (!m->G2) return fail(SEM_ERR_INVALID_ARG, "mesh built without SEM_GEOM_PAIR");
    switch (m->N) {
#define SEM_PAIR_CASE(n) \
    case n: return launch_pair_n<n, CG>(m, u, w, cg, st);
        SEM_PAIR_CASE(1) SEM_PAIR_CASE(2) SEM_PAIR_CASE(3) SEM_PAIR_CASE(4) SEM_PAIR_CASE(5)
        SEM_PAIR_CASE(6) SEM_PAIR_CASE(7) SEM_PAIR_CASE(8) SEM_PAIR_CASE(9) SEM_PAIR_CASE(10) SEM_PAIR_CASE(11)
#undef SEM_PAIR_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
}

int ax_launch_pair(const sem_mesh *m, const double *u, double *w, cudaStream_t st) {
    const CgFuse<double> none{};
    return dispatch_pair<false>(m, u, w, none, st);
}

int ax_cg_launch_pair(const sem_mesh *m, const CgFuse<double> &cg, double *w, cudaStream_t st) {
    return dispatch_pair<true>(m, nullptr, w, cg, st);
}

}  // namespace sem
