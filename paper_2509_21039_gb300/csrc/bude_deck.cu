// Deck preparation kernels: validation, ligand-type compaction and the
// type-pair parameter tables (the per-pair lookup of Eq. 3, built once per
// deck instead of once per pair).
#include "bude_internal.h"

namespace bude {

enum : unsigned {
    kErrType = 1u,      // an atom type outside [0, n_types)
    kErrCoord = 2u,     // a non-finite atom coordinate
    kErrForceField = 4u // radius <= 0, a non-finite parameter or a bad hbtype
};

__global__ void pack_protein_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                    int n, int n_types, unsigned* err)
{
    unsigned bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 a = src[i];
        int t = __float_as_int(a.w);
        if (t < 0 || t >= n_types) bad |= kErrType;
        if (!isfinite(a.x) || !isfinite(a.y) || !isfinite(a.z)) bad |= kErrCoord;
        dst[i] = a;
    }
    if (bad) atomicOr(err, bad);
}

// Single CTA: forcefield checks, ligand row map and the three pair tables.
__global__ void build_tables_kernel(const float4* __restrict__ lig_src, int n_lig,
                                    const float4* __restrict__ ff, int n_types,
                                    float4* __restrict__ lig_dst, PairF* __restrict__ tabF,
                                    PairG* __restrict__ tabG, PairD* __restrict__ tabD,
                                    int* __restrict__ row_type, int* n_rows_out, unsigned* err)
{
    __shared__ int s_row[BUDE_MAX_TYPES];   // type -> row, -1 unused
    __shared__ int s_type[BUDE_MAX_TYPES];  // row -> type
    __shared__ int s_nrows;
    __shared__ unsigned s_err;
    if (threadIdx.x == 0) { s_err = 0; s_nrows = 0; }
    for (int t = threadIdx.x; t < n_types; t += blockDim.x) s_row[t] = -1;
    __syncthreads();

    unsigned bad = 0;
    for (int t = threadIdx.x; t < n_types; t += blockDim.x) {
        float4 f = ff[t];
        int hb = __float_as_int(f.w);
        if (!(f.x > 0.f) || !isfinite(f.x) || !isfinite(f.y) || !isfinite(f.z) || hb < 0 || hb > 2)
            bad |= kErrForceField;
    }
    for (int l = threadIdx.x; l < n_lig; l += blockDim.x) {
        float4 a = lig_src[l];
        int t = __float_as_int(a.w);
        if (t < 0 || t >= n_types) {
            bad |= kErrType;
        } else {
            s_row[t] = 1;  // benign race: every writer stores the same value
        }
        if (!isfinite(a.x) || !isfinite(a.y) || !isfinite(a.z)) bad |= kErrCoord;
    }
    if (bad) atomicOr(&s_err, bad);
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = 0;
        for (int t = 0; t < n_types; ++t) {
            if (s_row[t] == 1) { s_type[r] = t; s_row[t] = r; ++r; }
            else s_row[t] = -1;
        }
        s_nrows = r;
        *n_rows_out = r;
        if (s_err) atomicOr(err, s_err);
    }
    __syncthreads();
    if (s_err) return;
    for (int l = threadIdx.x; l < n_lig; l += blockDim.x) {
        float4 a = lig_src[l];
        a.w = __int_as_float(s_row[__float_as_int(a.w)]);
        lig_dst[l] = a;
    }
    const int rows = s_nrows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) row_type[r] = s_type[r];
    for (int i = threadIdx.x; i < rows * n_types; i += blockDim.x) {
        const int ta = s_type[i / n_types], tb = i % n_types;
        const float4 fa = ff[ta], fb = ff[tb];
        const int ha = __float_as_int(fa.w), hb = __float_as_int(fb.w);
        // combination rules, evaluated in FP64 and rounded once
        const double R = (double)fa.x + (double)fb.x;
        const double H = 0.5 * ((double)fa.y + (double)fb.y);
        const double w = ((ha == 1 && hb == 2) || (ha == 2 && hb == 1)) ? 2.0 : 1.0;
        const double cE = kKE * (double)fa.z * (double)fb.z * w;
        const double S = ((ha != 0) != (hb != 0)) ? kKD : 0.0;
        const double inv_r = 1.0 / R;
        const double sh = sqrt(fabs(H));
        PairD d;
        d.sa = sh / R;
        d.sb = copysign(sh, H);
        d.ce = R / kDE + 1.0;
        d.ke1 = -2.0 * cE;
        d.ke0 = 3.0 * cE;
        d.cd = R / kDD + 1.0;
        d.kd1 = -2.0 * S;
        d.kd0 = 3.0 * S;
        tabD[i] = d;
        PairF f;
        f.inv_r = (float)inv_r; f.h = (float)H; f.ce = (float)d.ce; f.ke1 = (float)d.ke1;
        f.ke0 = (float)d.ke0; f.cd = (float)d.cd; f.kd1 = (float)d.kd1; f.kd0 = (float)d.kd0;
        tabF[i] = f;
        PairG g;
        g.inv_r = f.inv_r; g.h = f.h; g.ce = f.ce; g.ke1 = f.ke1;
        g.ke0 = f.ke0; g.cd = f.cd; g.kd1 = f.kd1; g.kd0 = f.kd0;
        g.hs = (float)(-2.0 * H * inv_r);
        g.ae1 = (float)(-3.0 / kDE * d.ke1);
        g.ae0 = (float)(-2.0 / kDE * d.ke0);
        g.ad1 = (float)(-3.0 / kDD * d.kd1);
        g.ad0 = (float)(-2.0 / kDD * d.kd0);
        g.sa = (float)(sh * inv_r);
        g.sb = (float)sh;
        g.pad = 0.f;
        tabG[i] = g;
    }
}

// Single CTA: stable sort of the protein atoms by type (a counting sort done
// one present type at a time with block-wide ballots), so that atoms of one
// type are consecutive.  The energy is a sum over atoms, so the order is
// free; the forcefield-gradient kernel relies on the runs.  Atoms with an
// invalid type are dropped here and reported by pack_protein_kernel.
__global__ void sort_protein_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                    int n, int n_types)
{
    __shared__ int s_count[BUDE_MAX_TYPES];
    __shared__ int s_warp[32];
    __shared__ int s_base, s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    for (int t = tid; t < n_types; t += blockDim.x) s_count[t] = 0;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        const int t = __float_as_int(src[i].w);
        if (t >= 0 && t < n_types) atomicAdd(&s_count[t], 1);
    }
    __syncthreads();
    for (int t = 0; t < n_types; ++t) {
        if (s_count[t] == 0) continue;  // uniform: every thread reads the same count
        for (int base = 0; base < n; base += blockDim.x) {
            const int i = base + tid;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            bool f = false;
            if (i < n) {
                a = src[i];
                f = __float_as_int(a.w) == t;
            }
            const unsigned m = __ballot_sync(0xffffffffu, f);
            const int before = __popc(m & ((1u << lane) - 1u));
            if (lane == 0) s_warp[warp] = __popc(m);
            __syncthreads();
            if (warp == 0) {
                int v = lane < nwarps ? s_warp[lane] : 0;
                int incl = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                if (lane < nwarps) s_warp[lane] = incl - v;  // exclusive prefix
                if (lane == 31) s_total = incl;              // block total (nwarps <= 32)
            }
            __syncthreads();
            if (f) dst[s_base + s_warp[warp] + before] = a;
            __syncthreads();
            if (tid == 0) s_base += s_total;
            __syncthreads();
        }
    }
}

// Single CTA: the midpoint c of the protein's bounding box, and the copy
// p - c of every atom, rounded once to FP32, with its type kept.  The FP32
// kernels work in this frame (they subtract c from the pose translations):
// the energy only depends on differences x' - p, and small coordinates keep
// the rounding of x' and of the squared distance small wherever the deck
// sits.  min and max are exact and order-free, so c is the same on every
// run.  n >= 1.
__global__ void recentre_protein_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                        int n, float* __restrict__ centre)
{
    __shared__ float s_lo[3][32], s_hi[3][32];
    __shared__ float s_c[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    for (int i = tid; i < n; i += blockDim.x) {
        const float4 a = src[i];
        lo[0] = fminf(lo[0], a.x); hi[0] = fmaxf(hi[0], a.x);
        lo[1] = fminf(lo[1], a.y); hi[1] = fmaxf(hi[1], a.y);
        lo[2] = fminf(lo[2], a.z); hi[2] = fmaxf(hi[2], a.z);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
        if (lane == 0) { s_lo[j][warp] = lo[j]; s_hi[j][warp] = hi[j]; }
    }
    __syncthreads();
    if (tid < 3) {
        float l = s_lo[tid][0], h = s_hi[tid][0];
        for (int w = 1; w < nwarps; ++w) { l = fminf(l, s_lo[tid][w]); h = fmaxf(h, s_hi[tid][w]); }
        float c = 0.5f * l + 0.5f * h;
        // a deck with a non-finite coordinate is rejected by the validation
        // pass; keep its frame finite meanwhile
        if (!isfinite(c)) c = 0.f;
        s_c[tid] = c;
        centre[tid] = c;
    }
    __syncthreads();
    const float cx = s_c[0], cy = s_c[1], cz = s_c[2];
    for (int i = tid; i < n; i += blockDim.x) {
        const float4 a = src[i];
        dst[i] = make_float4(a.x - cx, a.y - cy, a.z - cz, a.w);
    }
}

// Number of atoms whose type is polar (hbtype != 0).  A pair has a
// desolvation term exactly when one of its two atoms is polar, so these two
// counts give a deck's share of such pairs (its cost per pair iteration in a
// batched launch).  Atoms with an invalid type are not counted (the deck is
// rejected by the validation word anyway).
__global__ void count_polar_kernel(const float4* __restrict__ atoms, int n,
                                   const float4* __restrict__ ff, int n_types, int* __restrict__ count)
{
    int local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = __float_as_int(atoms[i].w);
        if (t >= 0 && t < n_types && __float_as_int(ff[t].w) != 0) ++local;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

cudaError_t launch_count_polar(const float4* atoms, int n, const float4* ff, int n_types,
                               int* count, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    count_polar_kernel<<<blocks, 256, 0, s>>>(atoms, n, ff, n_types, count);
    return cudaGetLastError();
}

cudaError_t launch_recentre_protein(const float4* src, float4* dst, int n, float* centre,
                                    cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    recentre_protein_kernel<<<1, 1024, 0, s>>>(src, dst, n, centre);
    return cudaGetLastError();
}

cudaError_t launch_pack_protein(const float4* src, float4* dst, int n, int n_types,
                                unsigned* err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    // validation pass (its copy is overwritten by the sorted one)
    pack_protein_kernel<<<blocks, 256, 0, s>>>(src, dst, n, n_types, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sort_protein_kernel<<<1, 1024, 0, s>>>(src, dst, n, n_types);
    return cudaGetLastError();
}

cudaError_t launch_build_tables(const float4* lig_src, int n_lig, const float4* ff, int n_types,
                                float4* lig_dst, PairF* tabF, PairG* tabG, PairD* tabD,
                                int* row_type, int* n_rows, unsigned* err, cudaStream_t s)
{
    build_tables_kernel<<<1, 512, 0, s>>>(lig_src, n_lig, ff, n_types, lig_dst, tabF, tabG,
                                          tabD, row_type, n_rows, err);
    return cudaGetLastError();
}

}  // namespace bude
