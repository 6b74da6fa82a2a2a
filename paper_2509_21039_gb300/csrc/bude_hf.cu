// Two-electron part of the Hartree-Fock Fock matrix over s-type Gaussians
// (arxiv 2509.21039, Sec. 2.2, Listing 5; Table 4), written for GB300.
//
// G_ij = sum_kl D_kl [2 (ij|kl) - (ik|jl)] is built from the unique integrals
// (ij|kl), i >= j, k >= l, ij >= kl: each adds, weighted by its degeneracy
// (1/2 for i = j, for k = l and for ij = kl),
//   F_ij += 4 D_kl v   F_kl += 4 D_ij v
//   F_ik -= D_jl v     F_il -= D_jk v     F_jk -= D_il v     F_jl -= D_ik v
// (the six updates of Listing 5), and G = F + F^T.  Per plan the kernel set
// precomputes, for every atom pair and primitive pair, the Gaussian product
// p = x_a + x_b, P = (x_a A + x_b B)/p and K = c_a c_b N_a N_b
// exp(-x_a x_b |A-B|^2/p), and the Schwarz bound Q_ij = sqrt((ij|ij)); a
// quartet with Q_ij Q_kl below the caller's threshold is skipped.  The pairs
// are kept sorted by Q (descending), so for the pair of rank a the partners
// that survive the threshold are the ranks b < min(a + 1, c_a) for a count c_a
// found by binary search.  Each call turns the counts into a prefix sum and
// hands out the surviving quartets, and only those, one per thread: no lane
// idles on a screened quartet and no index is decoded with a square root.
// Primitive quartets then cost
//   (ab|cd) = K_ab K_cd 2 pi^(5/2) / (p q sqrt(p+q)) F0(p q / (p+q) |P-Q|^2)
// with F0(t) = sqrt(pi/t) erf(sqrt t) / 2.  With rho = p q / (p+q) this is
//   K'_ab K'_cd sqrt(rho) erf(x) / x,   x = sqrt(rho) |P-Q|,
//   K' = K pi^(3/2) p^(-3/2),   sqrt(rho) = 1 / sqrt(1/p + 1/q),
// so a primitive quartet costs two reciprocal roots and an erf, with no
// division; the plan stores 1/p and K' per primitive pair.  GB300's FP64 units are a small
// fraction of its FP32 ones, so besides the FP64 kernel there is one that
// evaluates the primitive integrals in FP32 and accumulates the Fock matrix
// in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bude_internal.h"

namespace bude {

constexpr double kPi = 3.14159265358979323846;

// FP32 integrals take erf(x)/x, x = sqrt(t), from a table instead of erff:
// with F_k(t) = int_0^1 u^2k exp(-t u^2) du (the Boys functions, F_0(t) =
// (sqrt(pi)/2) erf(sqrt t)/sqrt t, dF_k/dt = -F_(k+1)), its Taylor expansion
// about the nearest grid point t_i = i/16,
//   erf(x)/x = (2/sqrt(pi)) sum_k F_k(t_i) (t_i - t)^k / k!,  k = 0..3,
// leaves at most (1/32)^4/4! F_4 < 5e-9 for |t - t_i| <= 1/32, 3e-8 of the
// smallest value on the grid.  Beyond t = 32, erf(sqrt t) is 1 to FP32
// precision (erfc(sqrt 32) < 2e-15) and erf(x)/x = 1/sqrt(t).  The grid
// values are computed once per plan on the host in FP64 from the series
// F_k(t) = exp(-t) sum_j (2t)^j / ((2k+1)(2k+3)...(2k+2j+1)), whose terms are
// all positive.
constexpr int kBoysPerUnit = 16;
constexpr int kBoysTmax = 32;
constexpr int kBoysN = kBoysTmax * kBoysPerUnit + 1;
// The FP64 kernel's table: t_i = i/32 up to t = 36 (erfc(6) < 2.2e-17, so
// erf(x)/x = 1/sqrt(t) in FP64 beyond it) and six Taylor terms: at most
// (1/64)^6/6! F_6 < 1.6e-15, 9e-15 of the smallest value on the grid.
constexpr int kBoys64PerUnit = 32;
constexpr int kBoys64Tmax = 36;
constexpr int kBoys64N = kBoys64Tmax * kBoys64PerUnit + 1;
constexpr int kBoys64Terms = 6;

// (2/sqrt(pi)) (-1)^k F_k(t) / k!, k < terms: the Horner coefficients of
// erf(x)/x in d = t' - t about t.
void boys_coefficients(double t, int terms, double* c)
{
    const double two_over_sqrt_pi = 2.0 / std::sqrt(kPi);
    double fact = 1.0;
    for (int k = 0; k < terms; ++k) {
        double term = 1.0 / (2 * k + 1), sum = term;
        for (int j = 1; j < 600; ++j) {
            term *= 2.0 * t / (2 * k + 2 * j + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        if (k > 0) fact *= k;
        c[k] = ((k & 1) ? -1.0 : 1.0) * two_over_sqrt_pi * std::exp(-t) * sum / fact;
    }
}

void boys_table(std::vector<float4>& tab)
{
    tab.resize(kBoysN);
    for (int i = 0; i < kBoysN; ++i) {
        double c[4];
        boys_coefficients((double)i / kBoysPerUnit, 4, c);
        tab[(size_t)i] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]);
    }
}

void boys_table64(std::vector<double2>& tab)
{
    tab.resize((size_t)kBoys64N * 3);
    for (int i = 0; i < kBoys64N; ++i) {
        double c[kBoys64Terms];
        boys_coefficients((double)i / kBoys64PerUnit, kBoys64Terms, c);
        for (int h = 0; h < 3; ++h) tab[(size_t)i * 3 + h] = make_double2(c[2 * h], c[2 * h + 1]);
    }
}

struct HfPlanDev {
    int n, ng;
    long long m;          // unique pairs n(n+1)/2
    const double4_32a* pq;    // [m][ng*ng] {Px, Py, Pz, 1/p}
    const double* kp;     // [m][ng*ng] K' = K pi^(3/2) p^(-3/2)
    const float4* pqf;    // FP32 copies
    const float* kpf;
    const double* schwarz;  // [m]
    const int2* pairs;      // [m] (i, j), i >= j
    const int* order;       // [m] pair index by rank of Q, largest first
    const double* qsorted;  // [m] Q by rank
    // the primitive products again, by rank and primitive-pair-major
    // ([ng*ng][m]), so that the lanes of a warp, which hold consecutive ranks,
    // read adjacent words
    const double4_32a* rpq;
    const double* rkp;
    const float4* rpqf;
    const float* rkpf;
    const int2* rpairs;     // [m] (i, j) of the pair of each rank
    const float4* boys;     // [kBoysN] FP32 integrals' table of erf(x)/x (below)
    const double2* boys64;  // [kBoys64N][3] the FP64 kernel's
};

__device__ __forceinline__ void pair_of(long long ij, int* i, int* j)
{
    long long a = (long long)((sqrt(8.0 * (double)ij + 1.0) - 1.0) * 0.5);
    while (a * (a + 1) / 2 > ij) --a;
    while ((a + 1) * (a + 2) / 2 <= ij) ++a;
    *i = (int)a;
    *j = (int)(ij - a * (a + 1) / 2);
}

// Gaussian products of every atom pair (i >= j) and primitive pair.
__global__ void hf_pairs_kernel(int n, int ng, const double* __restrict__ geom,
                                const double* __restrict__ xpnt, const double* __restrict__ coef,
                                double4_32a* __restrict__ pq, double* __restrict__ kp,
                                float4* __restrict__ pqf, float* __restrict__ kpf)
{
    const long long m = (long long)n * (n + 1) / 2;
    const int g2 = ng * ng;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m * g2;
         e += (long long)gridDim.x * blockDim.x) {
        const long long ij = e / g2;
        const int ab = (int)(e % g2), a = ab / ng, b = ab % ng;
        int i, j;
        pair_of(ij, &i, &j);
        const double xa = xpnt[a], xb = xpnt[b], p = xa + xb;
        double r2 = 0.0, P[3];
        for (int d = 0; d < 3; ++d) {
            const double A = geom[3 * i + d], B = geom[3 * j + d];
            r2 += (A - B) * (A - B);
            P[d] = (xa * A + xb * B) / p;
        }
        const double na = pow(2.0 * xa / kPi, 0.75), nb = pow(2.0 * xb / kPi, 0.75);
        const double K = coef[a] * coef[b] * na * nb * exp(-xa * xb * r2 / p);
        const double Kp = K * pow(kPi / p, 1.5);
        pq[e] = make_double4_32a(P[0], P[1], P[2], 1.0 / p);
        kp[e] = Kp;
        pqf[e] = make_float4((float)P[0], (float)P[1], (float)P[2], (float)(1.0 / p));
        kpf[e] = (float)Kp;
    }
}

// erf(x) / x from x^2, finite at x = 0 (2 / sqrt(pi)): the argument is
// floored far below any x^2 that matters, where erf(x) = 2x/sqrt(pi) to full
// precision, so that both reciprocal roots stay finite.
__device__ __forceinline__ double erf_over_x(double x2)
{
    const double y = fmax(x2, 1e-300);
    const double r = rsqrt(y);
    return erf(y * r) * r;
}
// 1/sqrt(x) for a positive normal float by the approximate reciprocal root
// with subnormals flushed: every argument here (1/p + 1/q of primitive
// exponents, or t >= 32) is a normal number, where this is the same MUFU
// operation as rsqrtf without the scaling rsqrtf wraps around it for
// subnormal inputs.
__device__ __forceinline__ float rsqrt_normal(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// erf(x)/x from x^2 = t by the table above (tab in shared memory): round 16 t
// to the nearest grid index with the 1.5 2^23 shift, so that the index is in
// the low mantissa bits and the grid point is exact, then three FMAs; past
// the table's end, 1/sqrt(t).  Both sides are computed and one selected:
// most warps hold primitives on both sides, and branching on the side (as
// the FP64 form below does) measured 3.55 -> 5.31 ms for 256 atoms.
__device__ __forceinline__ float erf_over_x(float t, const float4* __restrict__ tab, unsigned)
{
    constexpr float kShift = 12582912.f;   // 1.5 * 2^23: its ulp is 1
    const float tc = fminf(t, (float)kBoysTmax);
    const float y = fmaf(tc, (float)kBoysPerUnit, kShift);
    const int i = __float_as_int(y) - __float_as_int(kShift);
    const float d = fmaf(y - kShift, -1.f / kBoysPerUnit, tc);
    const float4 c = tab[i];
    const float f = fmaf(fmaf(fmaf(c.w, d, c.z), d, c.y), d, c.x);
    return t < (float)kBoysTmax ? f : rsqrt_normal(t);
}
// The same in FP64 with the finer table (read through the L1 cache: 55 KB),
// the 1.5 2^52 shift and five FMAs.  Each side runs only when a lane of
// `act` (the lanes calling together) needs it: on the FP64 pipe, which bounds
// this kernel, the warps whose primitives all lie on one side save the other
// side's operations (128 atoms 8.09 -> 7.92 ms, 256 atoms 194.9 -> 190.4 ms).
__device__ __forceinline__ double erf_over_x(double t, const double2* __restrict__ tab, unsigned act)
{
    constexpr double kShift = 6755399441055744.0;   // 1.5 * 2^52: its ulp is 1
    const bool near = t < (double)kBoys64Tmax;
    double f = 0.0;
    if (__any_sync(act, near)) {
        const double tc = fmin(t, (double)kBoys64Tmax);
        const double y = fma(tc, (double)kBoys64PerUnit, kShift);
        const long long i = __double_as_longlong(y) - __double_as_longlong(kShift);
        const double d = fma(y - kShift, -1.0 / kBoys64PerUnit, tc);
        const double2 c01 = __ldg(tab + 3 * i), c23 = __ldg(tab + 3 * i + 1),
                      c45 = __ldg(tab + 3 * i + 2);
        f = fma(c45.y, d, c45.x);
        f = fma(f, d, c23.y);
        f = fma(f, d, c23.x);
        f = fma(f, d, c01.y);
        f = fma(f, d, c01.x);
    }
    if (__any_sync(act, !near)) {
        const double g = rsqrt(t);
        f = near ? f : g;
    }
    return f;
}

// Precision-matched helpers for the template below (declared before it, so
// that the float instantiation never promotes to double).
__device__ __forceinline__ float hf_rsqrt(float x) { return rsqrt_normal(x); }
__device__ __forceinline__ double hf_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float hf_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double hf_fma(double a, double b, double c) { return fma(a, b, c); }

// Contracted (ij|kl) from the two pairs' primitive products.
template <typename T, typename T4>
__device__ __forceinline__ T contracted(const T4* __restrict__ A, const T4* __restrict__ C,
                                        const T* __restrict__ KA, const T* __restrict__ KC, int g2)
{
    T v = 0;
    for (int ab = 0; ab < g2; ++ab) {
        const T4 a = A[ab];
        const T ka = KA[ab];
        T w = 0;
        for (int cd = 0; cd < g2; ++cd) {
            const T4 c = C[cd];
            const T dx = a.x - c.x, dy = a.y - c.y, dz = a.z - c.z;
            const T r2 = hf_fma(dz, dz, hf_fma(dy, dy, dx * dx));
            const T rs = hf_rsqrt(a.w + c.w);   // sqrt(rho)
            w = hf_fma(KC[cd] * rs, erf_over_x(r2 * rs * rs), w);
        }
        v = hf_fma(ka, w, v);
    }
    return v;
}

// The same over the rank-ordered copies: primitive pair ab of rank a is at
// [ab * m + a].  G2 > 0: that many primitive pairs, known at compile time,
// with the partner's G2 products loaded up front (all in flight at once) and
// kept in registers across the loop over ab, whose body is unrolled over cd;
// G2 = 0: g2 at run time.
template <typename T, typename T4, int G2, typename TAB>
__device__ __forceinline__ T contracted_ranked(const T4* __restrict__ pq, const T* __restrict__ kp,
                                               long long m, long long a, long long b, int g2,
                                               const TAB* __restrict__ tab)
{
    // the lanes evaluating quartets together (the last items of a warp's
    // range may leave some out); every one of them runs the same loops below
    const unsigned act = __activemask();
    if constexpr (G2 > 0) {
        T4 c[G2];
        T kc[G2];
#pragma unroll
        for (int cd = 0; cd < G2; ++cd) {
            c[cd] = pq[cd * m + b];
            kc[cd] = kp[cd * m + b];
        }
        T v = 0;
        // the loop over ab stays rolled: unrolled, its G2^2 inlined erf
        // evaluations overflowed the instruction cache (ncu: warps stalled on
        // instruction fetch more than on anything else)
#pragma unroll 1
        for (int ab = 0; ab < G2; ++ab) {
            const T4 x = pq[ab * m + a];
            const T ka = kp[ab * m + a];
            T w = 0;
#pragma unroll
            for (int cd = 0; cd < G2; ++cd) {
                const T dx = x.x - c[cd].x, dy = x.y - c[cd].y, dz = x.z - c[cd].z;
                const T r2 = hf_fma(dz, dz, hf_fma(dy, dy, dx * dx));
                const T rs = hf_rsqrt(x.w + c[cd].w);   // sqrt(rho)
                w = hf_fma(kc[cd] * rs, erf_over_x(r2 * rs * rs, tab, act), w);
            }
            v = hf_fma(ka, w, v);
        }
        return v;
    }
    T v = 0;
    for (int ab = 0; ab < g2; ++ab) {
        const T4 x = pq[ab * m + a];
        const T ka = kp[ab * m + a];
        T w = 0;
        for (int cd = 0; cd < g2; ++cd) {
            const T4 c = pq[cd * m + b];
            const T dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
            const T r2 = hf_fma(dz, dz, hf_fma(dy, dy, dx * dx));
            const T rs = hf_rsqrt(x.w + c.w);   // sqrt(rho)
            w = hf_fma(kp[cd * m + b] * rs, erf_over_x(r2 * rs * rs, tab, act), w);
        }
        v = hf_fma(ka, w, v);
    }
    return v;
}

// The FP32 form of contracted_ranked for G2 >= 2 on packed FP32x2
// instructions (Blackwell's FADD2/FMUL2/FFMA2): the partner's primitive pairs
// go in twos, so one instruction serves two primitive integrals wherever
// their operands pair up (distances, exponent sums, t, the grid offsets and
// the prefactors); the table reads, the Horner steps and the roots stay
// scalar.  The partner's coordinates are kept negated, so that x - c is one
// packed add with the same rounding.  Half the issue slots of the scalar
// loop's FP32 work; the two lanes' sums of each ab meet once at its end.
template <int G2>
__device__ __forceinline__ float contracted_ranked_x2(const float4* __restrict__ pq,
                                                      const float* __restrict__ kp, long long m,
                                                      long long a, long long b,
                                                      const float4* __restrict__ tab)
{
    constexpr int NP = G2 / 2;
    constexpr float kShift = 12582912.f;   // 1.5 * 2^23, as in erf_over_x
    float2 ncx[NP], ncy[NP], ncz[NP], cw[NP], ck[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float4 u = pq[(2 * k) * m + b], v = pq[(2 * k + 1) * m + b];
        ncx[k] = make_float2(-u.x, -v.x);
        ncy[k] = make_float2(-u.y, -v.y);
        ncz[k] = make_float2(-u.z, -v.z);
        cw[k] = make_float2(u.w, v.w);
        ck[k] = make_float2(kp[(2 * k) * m + b], kp[(2 * k + 1) * m + b]);
    }
    float4 cl = make_float4(0.f, 0.f, 0.f, 0.f);
    float kl = 0.f;
    if constexpr (G2 % 2) {
        cl = pq[(G2 - 1) * m + b];
        kl = kp[(G2 - 1) * m + b];
    }
    const float2 shift2 = make_float2(kShift, kShift);
    const float2 per2 = make_float2((float)kBoysPerUnit, (float)kBoysPerUnit);
    const float2 inv2 = make_float2(-1.f / kBoysPerUnit, -1.f / kBoysPerUnit);
    float v = 0.f;
    // rolled over ab, as in contracted_ranked (instruction cache)
#pragma unroll 1
    for (int ab = 0; ab < G2; ++ab) {
        const float4 x = pq[ab * m + a];
        const float ka = kp[ab * m + a];
        const float2 xx = make_float2(x.x, x.x), xy = make_float2(x.y, x.y);
        const float2 xz = make_float2(x.z, x.z), xw = make_float2(x.w, x.w);
        float2 w2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 dx = __fadd2_rn(xx, ncx[k]);
            const float2 dy = __fadd2_rn(xy, ncy[k]);
            const float2 dz = __fadd2_rn(xz, ncz[k]);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 sw = __fadd2_rn(xw, cw[k]);
            const float2 rs = make_float2(rsqrt_normal(sw.x), rsqrt_normal(sw.y));   // sqrt(rho)
            const float2 t = __fmul2_rn(__fmul2_rn(r2, rs), rs);
            // erf(x)/x of both, as erf_over_x: grid index and offset packed
            const float2 tc = make_float2(fminf(t.x, (float)kBoysTmax), fminf(t.y, (float)kBoysTmax));
            const float2 y = __ffma2_rn(tc, per2, shift2);
            const float2 d = __ffma2_rn(__fadd2_rn(y, make_float2(-kShift, -kShift)), inv2, tc);
            const float4 c0 = tab[__float_as_int(y.x) - __float_as_int(kShift)];
            const float4 c1 = tab[__float_as_int(y.y) - __float_as_int(kShift)];
            float2 f;
            f.x = fmaf(fmaf(fmaf(c0.w, d.x, c0.z), d.x, c0.y), d.x, c0.x);
            f.y = fmaf(fmaf(fmaf(c1.w, d.y, c1.z), d.y, c1.y), d.y, c1.x);
            f.x = t.x < (float)kBoysTmax ? f.x : rsqrt_normal(t.x);
            f.y = t.y < (float)kBoysTmax ? f.y : rsqrt_normal(t.y);
            w2 = __ffma2_rn(__fmul2_rn(ck[k], rs), f, w2);
        }
        float w = w2.x + w2.y;
        if constexpr (G2 % 2) {
            const float dx = x.x - cl.x, dy = x.y - cl.y, dz = x.z - cl.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rs = rsqrt_normal(x.w + cl.w);
            w = fmaf(kl * rs, erf_over_x(r2 * rs * rs, tab, 0u), w);
        }
        v = fmaf(ka, w, v);
    }
    return v;
}

// Gather of the primitive products into the rank-ordered copies.
__global__ void hf_rank_copy_kernel(const HfPlanDev P, double4_32a* __restrict__ rpq,
                                    double* __restrict__ rkp, float4* __restrict__ rpqf,
                                    float* __restrict__ rkpf)
{
    const int g2 = P.ng * P.ng;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P.m * g2;
         e += (long long)gridDim.x * blockDim.x) {
        const long long ab = e / P.m, a = e % P.m;
        const long long src = (long long)P.order[a] * g2 + ab;
        rpq[e] = P.pq[src];
        rkp[e] = P.kp[src];
        rpqf[e] = P.pqf[src];
        rkpf[e] = P.kpf[src];
    }
}

// (i, j) of the pair of every rank, once per plan.
__global__ void hf_rank_pairs_kernel(const HfPlanDev P, int2* __restrict__ rpairs)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < P.m;
         a += (long long)gridDim.x * blockDim.x)
        rpairs[a] = P.pairs[P.order[a]];
}

__device__ double contracted_f64(const HfPlanDev& P, long long ij, long long kl)
{
    const int g2 = P.ng * P.ng;
    return contracted<double, double4_32a>(P.pq + ij * g2, P.pq + kl * g2, P.kp + ij * g2,
                                           P.kp + kl * g2, g2);
}

// Schwarz bounds Q_ij = sqrt((ij|ij)) in FP64.
__global__ void hf_schwarz_kernel(const HfPlanDev P, double* __restrict__ q)
{
    for (long long ij = blockIdx.x * (long long)blockDim.x + threadIdx.x; ij < P.m;
         ij += (long long)gridDim.x * blockDim.x)
        q[ij] = sqrt(fabs(contracted_f64(P, ij, ij)));
}

// (i, j) of every pair, once per plan.
__global__ void hf_pair_table_kernel(long long m, int2* __restrict__ pairs)
{
    for (long long ij = blockIdx.x * (long long)blockDim.x + threadIdx.x; ij < m;
         ij += (long long)gridDim.x * blockDim.x) {
        int i, j;
        pair_of(ij, &i, &j);
        pairs[ij] = make_int2(i, j);
    }
}

// w[a] = number of surviving partners b <= a of the pair of rank a: the ranks
// b < c_a with Q_b Q_a >= tol (a prefix, Q being sorted descending), capped at
// a + 1 so that every unordered quartet is counted once.
__global__ void hf_count_kernel(const HfPlanDev P, double tol, long long* __restrict__ w)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < P.m;
         a += (long long)gridDim.x * blockDim.x) {
        const double qa = P.qsorted[a];
        long long lo = 0, hi = a + 1;  // count in [0, a + 1]
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (P.qsorted[mid] * qa >= tol) lo = mid + 1; else hi = mid;
        }
        w[a] = lo;
    }
}

// In-place exclusive prefix sum of w[0..m) into prefix[0..m] by one CTA of
// 1024 threads: each thread scans a contiguous slice, the slice totals are
// scanned in shared memory, and prefix[m] is the number of quartets.
__global__ void __launch_bounds__(1024) hf_scan_kernel(const long long* __restrict__ w, long long m,
                                                      long long* __restrict__ prefix)
{
    __shared__ long long s_tot[1024];
    const int t = threadIdx.x;
    const long long per = (m + blockDim.x - 1) / blockDim.x;
    const long long b0 = min(m, (long long)t * per), b1 = min(m, b0 + per);
    long long sum = 0;
    for (long long a = b0; a < b1; ++a) sum += w[a];
    s_tot[t] = sum;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const long long v = s_tot[k];
            s_tot[k] = run;
            run += v;
        }
        prefix[m] = run;
    }
    __syncthreads();
    long long run = s_tot[t];
    for (long long a = b0; a < b1; ++a) {
        prefix[a] = run;
        run += w[a];
    }
}

// One thread per surviving quartet: work item x lies in the rank a with
// prefix[a] <= x < prefix[a + 1] and pairs with rank b = x - prefix[a].  Each
// warp takes a contiguous range of about total / warps items, its lanes the
// items x = x0 + lane, x0 + lane + 32, ...: a lane finds its first rank by
// binary search and every later one by stepping forward from the last (the
// next item is 32 further on, mostly in the same or the next rank), instead
// of one search of about log2(m) dependent loads per item.  Consecutive
// lanes then mostly share the rank a, whose data are warp-uniform loads, and
// hold consecutive ranks b, whose data are adjacent words.
template <bool F32, int G2>
__global__ void __launch_bounds__(128, 1) hf_fock_kernel(const HfPlanDev P,
                                                      const long long* __restrict__ prefix,
                                                      const double* __restrict__ D,
                                                      double* __restrict__ F)
{
    const long long total = prefix[P.m];
    const int n = P.n;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long per = ((total + warps - 1) / warps + 31) & ~31ll;
    const long long x0 = warp * per, x1 = min(total, x0 + per);
    const int g2 = P.ng * P.ng;
    // FP32 integrals: the erf(x)/x table, staged once per CTA
    const float4* tab = nullptr;
    if constexpr (F32) {
        __shared__ float4 s_boys[kBoysN];
        for (int e = threadIdx.x; e < kBoysN; e += blockDim.x) s_boys[e] = P.boys[e];
        __syncthreads();
        tab = s_boys;
    }
    long long a = -1;
    for (long long x = x0 + lane; x < x1; x += 32) {
        if (a < 0) {
            long long lo = 0, hi = P.m - 1;  // largest a with prefix[a] <= x
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
            }
            a = lo;
        } else {
            while (prefix[a + 1] <= x) ++a;
        }
        const long long b = x - prefix[a];
        const int2 pij = P.rpairs[a], pkl = P.rpairs[b];
        const int i = pij.x, j = pij.y, k = pkl.x, l = pkl.y;
        double v;
        if constexpr (F32 && G2 >= 2)
            v = (double)contracted_ranked_x2<G2>(P.rpqf, P.rkpf, P.m, a, b, tab);
        else if constexpr (F32)
            v = (double)contracted_ranked<float, float4, G2>(P.rpqf, P.rkpf, P.m, a, b, g2, tab);
        else
            v = contracted_ranked<double, double4_32a, G2>(P.rpq, P.rkp, P.m, a, b, g2, P.boys64);
        if (i == j) v *= 0.5;
        if (k == l) v *= 0.5;
        if (a == b) v *= 0.5;
        // the six updates are symmetric under (ij) <-> (kl) once G = F + F^T.
        // A full warp on one (ij) adds its F_ij terms in registers first: 32
        // atomics on one address would serialise.
        const double cij = 4.0 * D[(size_t)k * n + l] * v;
        const unsigned act = __activemask();
        const long long a0 = __shfl_sync(act, a, 0);
        if (act == 0xffffffffu && __all_sync(act, a == a0)) {
            double t = cij;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) atomicAdd(F + (size_t)i * n + j, t);
        } else {
            atomicAdd(F + (size_t)i * n + j, cij);
        }
        atomicAdd(F + (size_t)k * n + l, 4.0 * D[(size_t)i * n + j] * v);
        atomicAdd(F + (size_t)i * n + k, -D[(size_t)j * n + l] * v);
        atomicAdd(F + (size_t)i * n + l, -D[(size_t)j * n + k] * v);
        atomicAdd(F + (size_t)j * n + k, -D[(size_t)i * n + l] * v);
        atomicAdd(F + (size_t)j * n + l, -D[(size_t)i * n + k] * v);
    }
}

// Two full waves of CTAs: the warps' item ranges are equal, and halving
// them shortens the end of the launch, where some warps of a CTA are done
// (measured at 256 atoms: one wave 5.31 ms, two 5.18 ms).  The kernel is
// built for one CTA per SM at least, which leaves the compiler its register
// choice (120 registers, 4 CTAs per SM): capping it at 64-80 registers for
// 6-8 CTAs per SM ran at 6.0-6.6 ms.
template <bool F32, int G2>
cudaError_t launch_fock_g(const HfPlanDev& P, const long long* prefix, const double* D, double* F,
                          int sms, cudaStream_t s)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hf_fock_kernel<F32, G2>, 128, 0);
    if (e != cudaSuccess) return e;
    hf_fock_kernel<F32, G2><<<(unsigned)(2 * sms * std::max(occ, 1)), 128, 0, s>>>(P, prefix, D, F);
    return cudaGetLastError();
}

template <bool F32>
cudaError_t launch_fock(const HfPlanDev& P, const long long* prefix, const double* D, double* F,
                        int sms, cudaStream_t s)
{
    switch (P.ng) {
    case 1: return launch_fock_g<F32, 1>(P, prefix, D, F, sms, s);
    case 2: return launch_fock_g<F32, 4>(P, prefix, D, F, sms, s);
    case 3: return launch_fock_g<F32, 9>(P, prefix, D, F, sms, s);
    default: return launch_fock_g<F32, 0>(P, prefix, D, F, sms, s);
    }
}

// G = F + F^T
__global__ void hf_symmetrise_kernel(const double* __restrict__ F, double* __restrict__ G, int n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        G[e] = F[(size_t)i * n + j] + F[(size_t)j * n + i];
    }
}

}  // namespace bude

using namespace bude;

struct bude_hf {
    int device = 0;
    int n = 0, ng = 0;
    long long m = 0;
    double* geom = nullptr;
    double* xc = nullptr;  // xpnt[ng], coef[ng]
    double4_32a* pq = nullptr;
    double* kp = nullptr;
    float4* pqf = nullptr;
    float* kpf = nullptr;
    double* schwarz = nullptr;
    double* fock = nullptr;  // [n][n] accumulation buffer
    int2* pairs = nullptr;       // [m]
    int* order = nullptr;        // [m]
    double* qsorted = nullptr;   // [m]
    long long* counts = nullptr; // [m] per-call survivor counts
    long long* prefix = nullptr; // [m + 1]
    double4_32a* rpq = nullptr;  // rank-ordered copies, [ng*ng][m]
    double* rkp = nullptr;
    float4* rpqf = nullptr;
    float* rkpf = nullptr;
    int2* rpairs = nullptr;      // [m]
    float4* boys = nullptr;      // [kBoysN]
    double2* boys64 = nullptr;   // [kBoys64N][3]
    HfPlanDev view() const
    {
        HfPlanDev v;
        v.n = n;
        v.ng = ng;
        v.m = m;
        v.pq = pq;
        v.kp = kp;
        v.pqf = pqf;
        v.kpf = kpf;
        v.schwarz = schwarz;
        v.pairs = pairs;
        v.order = order;
        v.qsorted = qsorted;
        v.rpq = rpq;
        v.rkp = rkp;
        v.rpqf = rpqf;
        v.rkpf = rkpf;
        v.rpairs = rpairs;
        v.boys = boys;
        v.boys64 = boys64;
        return v;
    }
};

extern "C" BUDE_API int bude_hf_destroy(bude_hf* h)
{
    Range range_("bude_hf_destroy");
    if (!h) return BUDE_OK;
    cudaDeviceSynchronize();
    cudaFree(h->geom);
    cudaFree(h->xc);
    cudaFree(h->pq);
    cudaFree(h->kp);
    cudaFree(h->pqf);
    cudaFree(h->kpf);
    cudaFree(h->schwarz);
    cudaFree(h->fock);
    cudaFree(h->pairs);
    cudaFree(h->order);
    cudaFree(h->qsorted);
    cudaFree(h->counts);
    cudaFree(h->prefix);
    cudaFree(h->rpq);
    cudaFree(h->rkp);
    cudaFree(h->rpqf);
    cudaFree(h->rkpf);
    cudaFree(h->rpairs);
    cudaFree(h->boys);
    cudaFree(h->boys64);
    delete h;
    return BUDE_OK;
}

extern "C" BUDE_API int bude_hf_create(int32_t n_atoms, const double* geom, int32_t ngauss,
                                       const double* xpnt, const double* coef, void* stream,
                                       bude_hf** out)
{
    Range range_("bude_hf_create");
    if (!out) return BUDE_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_atoms < 1 || ngauss < 1 || ngauss > 8 || !geom || !xpnt || !coef)
        return BUDE_ERR_INVALID_ARG;
    for (int a = 0; a < ngauss; ++a)
        if (!(xpnt[a] > 0.0) || !std::isfinite(xpnt[a]) || !std::isfinite(coef[a]))
            return BUDE_ERR_INVALID_ARG;
    for (long long e = 0; e < 3ll * n_atoms; ++e)
        if (!std::isfinite(geom[e])) return BUDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    bude_hf* h = new bude_hf;
    cudaGetDevice(&h->device);
    h->n = n_atoms;
    h->ng = ngauss;
    h->m = (long long)n_atoms * (n_atoms + 1) / 2;
    const size_t e = (size_t)h->m * ngauss * ngauss;
    auto bail = [&](int code) { bude_hf_destroy(h); return code; };
    if (dev_alloc((void**)&h->geom, 3 * sizeof(double) * n_atoms) ||
        dev_alloc((void**)&h->xc, 2 * sizeof(double) * ngauss) ||
        dev_alloc((void**)&h->pq, e * sizeof(double4_32a)) ||
        dev_alloc((void**)&h->kp, e * sizeof(double)) ||
        dev_alloc((void**)&h->pqf, e * sizeof(float4)) ||
        dev_alloc((void**)&h->kpf, e * sizeof(float)) ||
        dev_alloc((void**)&h->schwarz, (size_t)h->m * sizeof(double)) ||
        dev_alloc((void**)&h->fock, (size_t)n_atoms * n_atoms * sizeof(double)) ||
        dev_alloc((void**)&h->pairs, (size_t)h->m * sizeof(int2)) ||
        dev_alloc((void**)&h->order, (size_t)h->m * sizeof(int)) ||
        dev_alloc((void**)&h->qsorted, (size_t)h->m * sizeof(double)) ||
        dev_alloc((void**)&h->counts, (size_t)h->m * sizeof(long long)) ||
        dev_alloc((void**)&h->prefix, ((size_t)h->m + 1) * sizeof(long long)) ||
        dev_alloc((void**)&h->rpq, e * sizeof(double4_32a)) ||
        dev_alloc((void**)&h->rkp, e * sizeof(double)) ||
        dev_alloc((void**)&h->rpqf, e * sizeof(float4)) ||
        dev_alloc((void**)&h->rkpf, e * sizeof(float)) ||
        dev_alloc((void**)&h->rpairs, (size_t)h->m * sizeof(int2)) ||
        dev_alloc((void**)&h->boys, kBoysN * sizeof(float4)) ||
        dev_alloc((void**)&h->boys64, (size_t)kBoys64N * 3 * sizeof(double2)))
        return bail(BUDE_ERR_OOM);
    // host inputs: copied synchronously (plan creation is not on the hot path)
    std::vector<float4> boys;
    boys_table(boys);
    std::vector<double2> boys64;
    boys_table64(boys64);
    if (cudaMemcpy(h->boys, boys.data(), kBoysN * sizeof(float4), cudaMemcpyHostToDevice) ||
        cudaMemcpy(h->boys64, boys64.data(), boys64.size() * sizeof(double2), cudaMemcpyHostToDevice) ||
        cudaMemcpy(h->geom, geom, 3 * sizeof(double) * n_atoms, cudaMemcpyHostToDevice) ||
        cudaMemcpy(h->xc, xpnt, sizeof(double) * ngauss, cudaMemcpyHostToDevice) ||
        cudaMemcpy(h->xc + ngauss, coef, sizeof(double) * ngauss, cudaMemcpyHostToDevice))
        return bail(BUDE_ERR_CUDA);
    const long long blocks = std::min<long long>(4096, ((long long)e + 255) / 256);
    hf_pairs_kernel<<<(unsigned)std::max(1ll, blocks), 256, 0, s>>>(
        n_atoms, ngauss, h->geom, h->xc, h->xc + ngauss, h->pq, h->kp, h->pqf, h->kpf);
    const long long sb = std::min<long long>(4096, (h->m + 127) / 128);
    hf_schwarz_kernel<<<(unsigned)std::max(1ll, sb), 128, 0, s>>>(h->view(), h->schwarz);
    hf_pair_table_kernel<<<(unsigned)std::max(1ll, sb), 128, 0, s>>>(h->m, h->pairs);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return bail(BUDE_ERR_CUDA);
    // rank the pairs by their Schwarz bound, largest first (once per plan)
    {
        std::vector<double> q((size_t)h->m);
        if (cudaMemcpy(q.data(), h->schwarz, (size_t)h->m * sizeof(double), cudaMemcpyDeviceToHost))
            return bail(BUDE_ERR_CUDA);
        std::vector<int> ord((size_t)h->m);
        for (long long k = 0; k < h->m; ++k) ord[(size_t)k] = (int)k;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return q[x] > q[y]; });
        std::vector<double> qs((size_t)h->m);
        for (long long k = 0; k < h->m; ++k) qs[(size_t)k] = q[(size_t)ord[(size_t)k]];
        if (cudaMemcpy(h->order, ord.data(), (size_t)h->m * sizeof(int), cudaMemcpyHostToDevice) ||
            cudaMemcpy(h->qsorted, qs.data(), (size_t)h->m * sizeof(double), cudaMemcpyHostToDevice))
            return bail(BUDE_ERR_CUDA);
    }
    hf_rank_copy_kernel<<<(unsigned)std::max(1ll, blocks), 256, 0, s>>>(h->view(), h->rpq, h->rkp,
                                                                        h->rpqf, h->rkpf);
    hf_rank_pairs_kernel<<<(unsigned)std::max(1ll, sb), 128, 0, s>>>(h->view(), h->rpairs);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return bail(BUDE_ERR_CUDA);
    *out = h;
    return BUDE_OK;
}

extern "C" BUDE_API int bude_hf_quartets(bude_hf* h, double tol, int64_t* count, void* stream)
{
    Range range_("bude_hf_quartets");
    if (!h || !count || tol < 0.0 || !std::isfinite(tol)) return BUDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long cb = std::max(1ll, std::min<long long>(4096, (h->m + 255) / 256));
    hf_count_kernel<<<(unsigned)cb, 256, 0, s>>>(h->view(), tol, h->counts);
    hf_scan_kernel<<<1, 1024, 0, s>>>(h->counts, h->m, h->prefix);
    long long total = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&total, h->prefix + h->m, sizeof total, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return BUDE_ERR_CUDA;
    *count = total;
    return BUDE_OK;
}

extern "C" BUDE_API int bude_hf_fock(bude_hf* h, const double* dens, double* g, double tol,
                                     int32_t variant, void* stream)
{
    Range range_("bude_hf_fock");
    if (!h || !dens || !g || tol < 0.0 || !std::isfinite(tol)) return BUDE_ERR_INVALID_ARG;
    if (variant != BUDE_FP64 && variant != BUDE_FP32_IEEE) return BUDE_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nn = (size_t)h->n * h->n;
    if (cudaMemsetAsync(h->fock, 0, nn * sizeof(double), s) != cudaSuccess) return BUDE_ERR_CUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // surviving quartets: counts per rank, their prefix sum, then one thread each
    const long long cb = std::max(1ll, std::min<long long>(4096, (h->m + 255) / 256));
    hf_count_kernel<<<(unsigned)cb, 256, 0, s>>>(h->view(), tol, h->counts);
    hf_scan_kernel<<<1, 1024, 0, s>>>(h->counts, h->m, h->prefix);
    const cudaError_t le = variant == BUDE_FP64
                               ? launch_fock<false>(h->view(), h->prefix, dens, h->fock, sms, s)
                               : launch_fock<true>(h->view(), h->prefix, dens, h->fock, sms, s);
    if (le != cudaSuccess) return BUDE_ERR_CUDA;
    const long long sb = std::max(1ll, std::min<long long>(4096, ((long long)nn + 255) / 256));
    hf_symmetrise_kernel<<<(unsigned)sb, 256, 0, s>>>(h->fock, g, h->n);
    return cudaGetLastError() == cudaSuccess ? BUDE_OK : BUDE_ERR_CUDA;
}
