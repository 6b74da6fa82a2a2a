// Gradient of a weighted sum of pose energies, L = sum_k w_k E_k, with
// respect to the ligand atom coordinates and the per-type forcefield
// parameters (radius, hardness, elsc): what forcefield fitting and ligand
// design need from the scoring function.
//
// Same flat work space and shared-memory staging as the pose kernel, but
// every CTA only accumulates: there are no per-pose outputs, so no cross-CTA
// tile finish.  Per pair and pose the kernel needs, besides de/dd:
//   de/dR = -de/dd + hs w^2   (hs = -2H/R; the steric part of de/dd is hs w)
//   de/dH = w^2,   dphi_E = v_E^2 (3 - 2 v_E)
// summed with weight w_k/2 over the lane's poses for the current run of
// protein atoms of one type (the deck stores the protein sorted by type), and
// added per run into shared FP64 accumulators for the (ligand row, protein
// type) pair.  The ligand gradient R^T g is summed per ligand atom.  A second
// pass adds the CTAs' accumulators in CTA order and applies the combination
// rules (R = r_a + r_b, H = (h_a + h_b)/2, C_E = K_E q_a q_b w_ab).
#include <type_traits>

#include "bude_internal.h"

namespace bude {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int V, int P>
__global__ void param_kernel(const ParamArgs a)
{
    constexpr int TP = 32 * P;
    // even P: two poses per FP32x2 instruction, the pair record read once per
    // same-type run, and the desolvation terms left out on runs where S = 0
    constexpr bool PACK = P % 2 == 0;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int acc_lig = a.n_lig * 3;
    const int acc_len = acc_lig + a.n_rows * a.n_types * 3;
    double* s_acc = reinterpret_cast<double*>(smem);                        // [acc_len]
    size_t off = ((size_t)acc_len * sizeof(double) + 15) & ~size_t(15);
    float* s_tr = reinterpret_cast<float*>(smem + off);                     // [12][TP]
    float* s_w = s_tr + 12 * TP;                                            // [TP] w_k / 2
    off += (size_t)13 * TP * sizeof(float);
    PairG* s_pair = reinterpret_cast<PairG*>(smem + off);                   // [n_rows][n_types]
    off += (size_t)a.n_rows * a.n_types * sizeof(PairG);
    float4* s_pro = reinterpret_cast<float4*>(smem + off);                  // [chunk]

    const long long N = a.n_total;
    const long long C = gridDim.x;
    const long long c = blockIdx.x;
    long long x = c * N / C;
    const long long xe = (c + 1) * N / C;

    for (int i = threadIdx.x; i < acc_len; i += blockDim.x) s_acc[i] = 0.0;
    for (int i = threadIdx.x; i < a.n_rows * a.n_types; i += blockDim.x) s_pair[i] = a.pair[i];
    int staged_chunk = -1;
    const long long K = (long long)a.n_lig * a.n_pro;

    while (x < xe) {
        const long long t = x / K;
        const long long tile_k0 = t * K;
        const long long seg_end = xe < tile_k0 + K ? xe : tile_k0 + K;
        const long long pose0 = t * TP;
        __syncthreads();
        for (int s = threadIdx.x; s < TP; s += blockDim.x) {
            long long k = pose0 + s;
            const bool tail = k >= a.n_poses;
            if (tail) k = a.n_poses - 1;
            const long long n = a.n_poses;
            float sx, cx, sy, cy, sz, cz;
            if (V == kFAST) {
                __sincosf(a.poses[k], &sx, &cx);
                __sincosf(a.poses[n + k], &sy, &cy);
                __sincosf(a.poses[2 * n + k], &sz, &cz);
            } else {
                sincosf(a.poses[k], &sx, &cx);
                sincosf(a.poses[n + k], &sy, &cy);
                sincosf(a.poses[2 * n + k], &sz, &cz);
            }
            s_tr[0 * TP + s] = cy * cz;
            s_tr[1 * TP + s] = sx * sy * cz - cx * sz;
            s_tr[2 * TP + s] = cx * sy * cz + sx * sz;
            s_tr[3 * TP + s] = cy * sz;
            s_tr[4 * TP + s] = sx * sy * sz + cx * cz;
            s_tr[5 * TP + s] = cx * sy * sz - sx * cz;
            s_tr[6 * TP + s] = -sy;
            s_tr[7 * TP + s] = sx * cy;
            s_tr[8 * TP + s] = cx * cy;
            s_tr[9 * TP + s] = a.poses[3 * n + k] - a.ox;
            s_tr[10 * TP + s] = a.poses[4 * n + k] - a.oy;
            s_tr[11 * TP + s] = a.poses[5 * n + k] - a.oz;
            s_w[s] = tail ? 0.f : 0.5f * (a.weights ? a.weights[k] : 1.f);
        }
        __syncthreads();

        long long r0 = x - tile_k0;
        const long long r1 = seg_end - tile_k0;
        while (r0 < r1) {
            const int CL = a.chunk;
            const long long rowsK = (long long)a.n_lig * CL;
            const int q = (int)(r0 / rowsK);
            const long long cb = (long long)q * rowsK;
            const int len_q = min(CL, a.n_pro - q * CL);
            const long long cend = cb + (long long)a.n_lig * len_q;
            const long long sub_end = r1 < cend ? r1 : cend;
            if (q != staged_chunk) {
                __syncthreads();
                const float4* gsrc = a.pro + (size_t)q * CL;
                for (int i = threadIdx.x; i < len_q; i += blockDim.x) {
                    const float4 v = gsrc[i];
                    if constexpr (PACK) {
                        s_pro[2 * i] = make_float4(v.x, v.x, v.y, v.y);
                        s_pro[2 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
                    } else {
                        s_pro[i] = v;
                    }
                }
                __syncthreads();
                staged_chunk = q;
            }
            const long long len = sub_end - r0;
            long long i0 = r0 - cb + len * warp / W;
            const long long i1 = r0 - cb + len * (warp + 1) / W;
            int l = (int)(i0 / len_q);
            int p = (int)(i0 - (long long)l * len_q);
            float wv[P];
#pragma unroll
            for (int k = 0; k < P; ++k) wv[k] = s_w[lane + 32 * k];
            while (i0 < i1) {
                const long long row_base = (long long)l * len_q;
                const int pend = (int)((i1 - row_base) < len_q ? (i1 - row_base) : len_q);
                const float4 la = a.lig[l];
                const int row = __float_as_int(la.w);
                const volatile float* tr = s_tr;
                float xl[P], yl[P], zl[P], ngx[P], ngy[P], ngz[P];
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int s = lane + 32 * k;
                    xl[k] = tr[0 * TP + s] * la.x + tr[1 * TP + s] * la.y + tr[2 * TP + s] * la.z + tr[9 * TP + s];
                    yl[k] = tr[3 * TP + s] * la.x + tr[4 * TP + s] * la.y + tr[5 * TP + s] * la.z + tr[10 * TP + s];
                    zl[k] = tr[6 * TP + s] * la.x + tr[7 * TP + s] * la.y + tr[8 * TP + s] * la.z + tr[11 * TP + s];
                    ngx[k] = 0.f; ngy[k] = 0.f; ngz[k] = 0.f;
                }
                double* acc_row = s_acc + acc_lig + (size_t)row * a.n_types * 3;
                const PairG* prow = s_pair + (size_t)row * a.n_types;
                if constexpr (PACK) {
                    constexpr int H = P / 2;
                    // ng* accumulate f (p - x') = -dE/dx' per pose, two poses per pair
                    float2 nx[H], ny[H], nz[H], gx2[H], gy2[H], gz2[H], wv2[H];
#pragma unroll
                    for (int j = 0; j < H; ++j) {
                        nx[j] = make_float2(-xl[2 * j], -xl[2 * j + 1]);
                        ny[j] = make_float2(-yl[2 * j], -yl[2 * j + 1]);
                        nz[j] = make_float2(-zl[2 * j], -zl[2 * j + 1]);
                        gx2[j] = gy2[j] = gz2[j] = make_float2(0.f, 0.f);
                        wv2[j] = make_float2(wv[2 * j], wv[2 * j + 1]);
                    }
                    const float2 kmin2 = make_float2(kMinD2, kMinD2);
                    int pp = p;
                    while (pp < pend) {
                        const int tp = __float_as_int(s_pro[2 * pp + 1].z);
                        int run_end = pp + 1;
                        while (run_end < pend && __float_as_int(s_pro[2 * run_end + 1].z) == tp) ++run_end;
                        const PairG cp = prow[tp];
                        const float2 hs2 = make_float2(cp.hs, cp.hs);
                        const float2 ae1 = make_float2(cp.ae1, cp.ae1), ae0 = make_float2(cp.ae0, cp.ae0);
                        const float2 ad1 = make_float2(cp.ad1, cp.ad1), ad0 = make_float2(cp.ad0, cp.ad0);
                        // sums over the run: wv w^2, wv de/dd, wv v_E^2 (3 - 2 v_E); then
                        // de/dR = hs w^2 - de/dd gives the radius sum as hs sH - sD
                        float2 aH = make_float2(0.f, 0.f), aD = aH, aE = aH;
                        auto atom = [&](auto desolv_tag, int q2) {
                            constexpr bool DESOLV = decltype(desolv_tag)::value;
                            const float4 a0 = s_pro[2 * q2], a1 = s_pro[2 * q2 + 1];
                            const float2 px = make_float2(a0.x, a0.y), py = make_float2(a0.z, a0.w);
                            const float2 pz = make_float2(a1.x, a1.y);
#pragma unroll
                            for (int j = 0; j < H; ++j) {
                                const float2 dx = __fadd2_rn(px, nx[j]);
                                const float2 dy = __fadd2_rn(py, ny[j]);
                                const float2 dz = __fadd2_rn(pz, nz[j]);
                                float2 d2 = __ffma2_rn(dx, dx, kmin2);
                                d2 = __ffma2_rn(dy, dy, d2);
                                d2 = __ffma2_rn(dz, dz, d2);
                                const float2 y = make_float2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
                                const float2 d = (V == kFAST) ? __fmul2_rn(d2, y) : sqrt_rn_fma2(d2, y);
                                const float2 w = make_float2(clamp01(fmaf(d.x, -cp.inv_r, 1.f)),
                                                             clamp01(fmaf(d.y, -cp.inv_r, 1.f)));
                                const float2 ve = make_float2(clamp01(fmaf(d.x, -(float)(1.0 / kDE), cp.ce)),
                                                              clamp01(fmaf(d.y, -(float)(1.0 / kDE), cp.ce)));
                                float2 dedd = __fmul2_rn(hs2, w);
                                dedd = __ffma2_rn(ve, __ffma2_rn(ae1, ve, ae0), dedd);
                                if constexpr (DESOLV) {
                                    const float2 vd = make_float2(clamp01(fmaf(d.x, -(float)(1.0 / kDD), cp.cd)),
                                                                  clamp01(fmaf(d.y, -(float)(1.0 / kDD), cp.cd)));
                                    dedd = __ffma2_rn(vd, __ffma2_rn(ad1, vd, ad0), dedd);
                                }
                                const float2 f = __fmul2_rn(dedd, y);
                                gx2[j] = __ffma2_rn(f, dx, gx2[j]);
                                gy2[j] = __ffma2_rn(f, dy, gy2[j]);
                                gz2[j] = __ffma2_rn(f, dz, gz2[j]);
                                aH = __ffma2_rn(wv2[j], __fmul2_rn(w, w), aH);
                                aD = __ffma2_rn(wv2[j], dedd, aD);
                                const float2 t = __ffma2_rn(ve, make_float2(-2.f, -2.f), make_float2(3.f, 3.f));
                                aE = __ffma2_rn(__fmul2_rn(wv2[j], __fmul2_rn(ve, ve)), t, aE);
                            }
                        };
                        if (cp.ad1 != 0.f || cp.ad0 != 0.f) {
#pragma unroll 1
                            for (; pp < run_end; ++pp) atom(std::integral_constant<bool, true>(), pp);
                        } else {
#pragma unroll 1
                            for (; pp < run_end; ++pp) atom(std::integral_constant<bool, false>(), pp);
                        }
                        const float sH = warp_sum(aH.x + aH.y), sD = warp_sum(aD.x + aD.y);
                        const float sE = warp_sum(aE.x + aE.y);
                        if (lane == 0) {
                            atomicAdd(acc_row + tp * 3 + 0, (double)cp.hs * (double)sH - (double)sD);
                            atomicAdd(acc_row + tp * 3 + 1, (double)sH);
                            atomicAdd(acc_row + tp * 3 + 2, (double)sE);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < H; ++j) {
                        ngx[2 * j] = gx2[j].x; ngx[2 * j + 1] = gx2[j].y;
                        ngy[2 * j] = gy2[j].x; ngy[2 * j + 1] = gy2[j].y;
                        ngz[2 * j] = gz2[j].x; ngz[2 * j + 1] = gz2[j].y;
                    }
                } else {
                    float aR = 0.f, aH = 0.f, aE = 0.f;
                    int cur = -1;
                    for (int pp = p; pp < pend; ++pp) {
                        const float4 at = s_pro[pp];
                        const int tp = __float_as_int(at.w);
                        if (tp != cur) {  // warp-uniform: every lane reads the same atom
                            if (cur >= 0) {
                                const float sR = warp_sum(aR), sH = warp_sum(aH), sE = warp_sum(aE);
                                if (lane == 0) {
                                    atomicAdd(acc_row + cur * 3 + 0, (double)sR);
                                    atomicAdd(acc_row + cur * 3 + 1, (double)sH);
                                    atomicAdd(acc_row + cur * 3 + 2, (double)sE);
                                }
                            }
                            cur = tp;
                            aR = 0.f; aH = 0.f; aE = 0.f;
                        }
                        const PairG cp = prow[tp];
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const float dx = at.x - xl[k], dy = at.y - yl[k], dz = at.z - zl[k];
                            const float d2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, kMinD2)));
                            const float y = rsqrt_approx(d2);
                            const float d = (V == kFAST) ? d2 * y : sqrt_rn_fma(d2, y);
                            const float w = clamp01(fmaf(d, -cp.inv_r, 1.f));
                            const float ve = clamp01(fmaf(d, -(float)(1.0 / kDE), cp.ce));
                            const float vd = clamp01(fmaf(d, -(float)(1.0 / kDD), cp.cd));
                            float dedd = cp.hs * w;
                            dedd = fmaf(ve, fmaf(cp.ae1, ve, cp.ae0), dedd);
                            dedd = fmaf(vd, fmaf(cp.ad1, vd, cp.ad0), dedd);
                            const float f = dedd * y;
                            ngx[k] = fmaf(f, dx, ngx[k]);
                            ngy[k] = fmaf(f, dy, ngy[k]);
                            ngz[k] = fmaf(f, dz, ngz[k]);
                            const float w2 = w * w;
                            aR = fmaf(wv[k], fmaf(cp.hs, w2, -dedd), aR);
                            aH = fmaf(wv[k], w2, aH);
                            aE = fmaf(wv[k], ve * ve * fmaf(-2.f, ve, 3.f), aE);
                        }
                    }
                    if (cur >= 0) {
                        const float sR = warp_sum(aR), sH = warp_sum(aH), sE = warp_sum(aE);
                        if (lane == 0) {
                            atomicAdd(acc_row + cur * 3 + 0, (double)sR);
                            atomicAdd(acc_row + cur * 3 + 1, (double)sH);
                            atomicAdd(acc_row + cur * 3 + 2, (double)sE);
                        }
                    }
                }
                // dL/dx_l += sum_k (w_k/2) R_k^T g_k with g_k = -ng_k
                float v0 = 0.f, v1 = 0.f, v2 = 0.f;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int s = lane + 32 * k;
                    const float gx = -wv[k] * ngx[k], gy = -wv[k] * ngy[k], gz = -wv[k] * ngz[k];
                    v0 += tr[0 * TP + s] * gx + tr[3 * TP + s] * gy + tr[6 * TP + s] * gz;
                    v1 += tr[1 * TP + s] * gx + tr[4 * TP + s] * gy + tr[7 * TP + s] * gz;
                    v2 += tr[2 * TP + s] * gx + tr[5 * TP + s] * gy + tr[8 * TP + s] * gz;
                }
                v0 = warp_sum(v0);
                v1 = warp_sum(v1);
                v2 = warp_sum(v2);
                if (lane == 0) {
                    atomicAdd(s_acc + 3 * l + 0, (double)v0);
                    atomicAdd(s_acc + 3 * l + 1, (double)v1);
                    atomicAdd(s_acc + 3 * l + 2, (double)v2);
                }
                i0 = row_base + pend;
                ++l;
                p = 0;
            }
            r0 = sub_end;
        }
        x = seg_end;
    }
    __syncthreads();
    double* out = a.cta_acc + (size_t)c * acc_len;
    for (int i = threadIdx.x; i < acc_len; i += blockDim.x) out[i] = s_acc[i];
}

// Adds the CTAs' accumulators in CTA order: sums[i] = sum_c cta_acc[c][i].
// The loads of eight CTAs are issued before their sums (same order of
// additions), so that they are in flight together.
__global__ void param_sum_kernel(const double* __restrict__ cta_acc, int n_cta, int acc_len,
                                 double* __restrict__ sums)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < acc_len; i += gridDim.x * blockDim.x) {
        double v = 0.0;
        int c = 0;
        for (; c + 8 <= n_cta; c += 8) {
            double t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = cta_acc[(size_t)(c + u) * acc_len + i];
#pragma unroll
            for (int u = 0; u < 8; ++u) v += t[u];
        }
        for (; c < n_cta; ++c) v += cta_acc[(size_t)c * acc_len + i];
        sums[i] = v;
    }
}

// Chain rule from the (row, protein type) sums to per-type gradients: one
// CTA per type t (the last CTA copies the ligand gradients).  The CTA's
// threads split the (row, protein type) pairs in which t takes part, each
// summing its share in order, and the shares are added in a fixed order (a
// butterfly per warp, then the warps in order), so the result does not vary
// from call to call.  (One thread per type walking every pair in turn took
// 0.37 ms on the 64-atom deck: a chain of dependent loads.)
__global__ void __launch_bounds__(256) param_finish_kernel(
    const double* __restrict__ sums, int n_lig, int n_rows, int n_types,
    const int* __restrict__ row_type, const float4* __restrict__ ff, float* __restrict__ lig_grad,
    float* __restrict__ ff_grad)
{
    const int acc_lig = n_lig * 3;
    const int t = blockIdx.x;
    if (t >= n_types) {
        for (int i = threadIdx.x; i < acc_lig; i += blockDim.x) lig_grad[i] = (float)sums[i];
        return;
    }
    double gr = 0.0, gh = 0.0, gq = 0.0;
    const int pairs = n_rows * n_types;
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
        const int r = p / n_types, b = p - r * n_types;
        const int ta = row_type[r];
        const bool as_a = (ta == t), as_b = (b == t);
        if (!as_a && !as_b) continue;
        const double* v = sums + acc_lig + (size_t)p * 3;
        const float4 fa = ff[ta], fb = ff[b];
        const int ha = __float_as_int(fa.w), hb = __float_as_int(fb.w);
        const double wab = ((ha == 1 && hb == 2) || (ha == 2 && hb == 1)) ? 2.0 : 1.0;
        const double v0 = v[0], v1 = v[1], v2 = v[2];
        if (as_a) {
            gr += v0;
            gh += 0.5 * v1;
            gq += kKE * wab * (double)fb.z * v2;
        }
        if (as_b) {
            gr += v0;
            gh += 0.5 * v1;
            gq += kKE * wab * (double)fa.z * v2;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
        gh += __shfl_xor_sync(0xffffffffu, gh, o);
        gq += __shfl_xor_sync(0xffffffffu, gq, o);
    }
    __shared__ double s_w[3][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_w[0][w] = gr;
        s_w[1][w] = gh;
        s_w[2][w] = gq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0.0, r1 = 0.0, r2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            r0 += s_w[0][k];
            r1 += s_w[1][k];
            r2 += s_w[2][k];
        }
        ff_grad[3 * t + 0] = (float)r0;
        ff_grad[3 * t + 1] = (float)r1;
        ff_grad[3 * t + 2] = (float)r2;
    }
}

template __global__ void param_kernel<kIEEE, 1>(const ParamArgs);
template __global__ void param_kernel<kIEEE, 2>(const ParamArgs);
template __global__ void param_kernel<kIEEE, 4>(const ParamArgs);
template __global__ void param_kernel<kIEEE, 8>(const ParamArgs);
template __global__ void param_kernel<kFAST, 1>(const ParamArgs);
template __global__ void param_kernel<kFAST, 2>(const ParamArgs);
template __global__ void param_kernel<kFAST, 4>(const ParamArgs);
template __global__ void param_kernel<kFAST, 8>(const ParamArgs);

const void* kernel_param(int variant, int P)
{
    const bool fast = variant == kFAST;
    switch (P) {
    case 1: return fast ? (const void*)param_kernel<kFAST, 1> : (const void*)param_kernel<kIEEE, 1>;
    case 2: return fast ? (const void*)param_kernel<kFAST, 2> : (const void*)param_kernel<kIEEE, 2>;
    case 4: return fast ? (const void*)param_kernel<kFAST, 4> : (const void*)param_kernel<kIEEE, 4>;
    case 8: return fast ? (const void*)param_kernel<kFAST, 8> : (const void*)param_kernel<kIEEE, 8>;
    }
    return nullptr;
}

size_t param_smem_bytes(int P, int n_lig, int n_rows, int n_types, int chunk)
{
    const size_t TP = 32u * (size_t)P;
    const size_t acc = (size_t)(n_lig * 3 + n_rows * n_types * 3) * sizeof(double);
    size_t off = (acc + 15) & ~size_t(15);
    off += 13 * TP * sizeof(float);
    off += (size_t)n_rows * n_types * sizeof(PairG);
    return off + (size_t)chunk * param_atom_bytes(P);
}

cudaError_t launch_param_reduce(const double* cta_acc, int n_cta, int n_lig, int n_rows,
                                int n_types, double* sums, const int* row_type, const float4* ff,
                                float* lig_grad, float* ff_grad, cudaStream_t s)
{
    const int acc_len = n_lig * 3 + n_rows * n_types * 3;
    int blocks = (acc_len + 255) / 256;
    param_sum_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(cta_acc, n_cta, acc_len, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    param_finish_kernel<<<n_types + 1, 256, 0, s>>>(sums, n_lig, n_rows, n_types, row_type, ff,
                                                     lig_grad, ff_grad);
    return cudaGetLastError();
}

}  // namespace bude
