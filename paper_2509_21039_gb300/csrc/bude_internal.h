// Internal declarations shared by the host API and the kernel translation
// units of libbude.so.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bude.h"
#include "bude_kernels.cuh"

namespace bude {

// Every device allocation of the library goes through dev_alloc, so that a
// test can make the n-th one fail (bude_debug_fail_alloc) and check that each
// error path releases what it took.  An injected failure returns
// cudaErrorMemoryAllocation without touching the CUDA context.
cudaError_t dev_alloc(void** p, size_t bytes);

// NVTX range around a public entry point (a no-op unless a profiler is
// attached).
struct Range {
    explicit Range(const char* name);
    ~Range();
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Kernel entry of pose_kernel<V, P, G>, or nullptr when that combination is
// not built.  Defined in the per-variant translation units.
const void* kernel_ieee(int P, bool G);
const void* kernel_fast(int P, bool G);
const void* kernel_comp(int P, bool G);
const void* kernel_f64(int P, bool G);
// pose_kernel<V, P, G, true>: energies or adjoint with cutoff culling (even P).
const void* kernel_ieee_cull(int P, bool G);
const void* kernel_fast_cull(int P, bool G);
const void* kernel_comp_cull(int P, bool G);

cudaError_t launch_pack_protein(const float4* src, float4* dst, int n, int n_types,
                                unsigned* err, cudaStream_t s);
// The midpoint of the protein's bounding box (centre[0..2]) and the copy
// dst = src - centre of every atom (types kept).
cudaError_t launch_recentre_protein(const float4* src, float4* dst, int n, float* centre,
                                    cudaStream_t s);
cudaError_t launch_count_polar(const float4* atoms, int n, const float4* ff, int n_types,
                               int* count, cudaStream_t s);
cudaError_t launch_build_tables(const float4* lig_src, int n_lig, const float4* ff, int n_types,
                                float4* lig_dst, PairF* tabF, PairG* tabG, PairD* tabD,
                                int* row_type, int* n_rows, unsigned* err, cudaStream_t s);

// Forcefield/ligand gradient kernel (bude_param.cu).
struct ParamArgs {
    const float4* pro;     // sorted by type, in the frame with origin (ox, oy, oz)
    const float4* lig;     // row-mapped
    const PairG* pair;     // [n_rows][n_types]
    const float* poses;    // [6][n_poses]
    const float* weights;  // [n_poses] or null (all ones)
    long long n_poses;
    long long n_total;     // tiles * n_lig * n_pro
    double* cta_acc;       // [grid][n_lig*3 + n_rows*n_types*3]
    int n_lig, n_pro, n_types, n_rows, chunk;
    float ox, oy, oz;      // subtracted from the pose translations (Instance::ox)
};
const void* kernel_param(int variant, int P);
// Shared-memory bytes per staged protein atom of param_kernel: the packed
// kernels (even P) duplicate each coordinate into both halves of an FP32x2 pair.
__host__ __device__ constexpr int param_atom_bytes(int P) { return P % 2 == 0 ? 32 : 16; }
size_t param_smem_bytes(int P, int n_lig, int n_rows, int n_types, int chunk);
cudaError_t launch_param_reduce(const double* cta_acc, int n_cta, int n_lig, int n_rows,
                                int n_types, double* sums, const int* row_type, const float4* ff,
                                float* lig_grad, float* ff_grad, cudaStream_t s);

cudaError_t launch_refine_init(float* alpha, long long n, float step0, cudaStream_t s);
cudaError_t launch_refine_propose(const float* p, const float* g, const float* alpha,
                                  float* trial, long long n, cudaStream_t s);
cudaError_t launch_refine_accept(float* p, float* E, float* g, const float* trial,
                                 const float* Et, const float* gt, float* alpha, long long n,
                                 float grow, float shrink, cudaStream_t s);

}  // namespace bude
