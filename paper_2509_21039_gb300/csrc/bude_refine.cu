// Element-wise kernels of the on-device pose refinement (bude_refine): the
// step proposal and the accept/reject update around each adjoint evaluation.
// Rule, per pose: p' = p - alpha g / |g| (p' = p when |g| is 0 or not
// finite); accept when E(p') < E(p), then alpha *= grow, else alpha *= shrink.
#include "bude_internal.h"

namespace bude {

__global__ void refine_init_kernel(float* __restrict__ alpha, long long n, float step0)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        alpha[k] = step0;
}

__global__ void refine_propose_kernel(const float* __restrict__ p, const float* __restrict__ g,
                                      const float* __restrict__ alpha, float* __restrict__ trial,
                                      long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        float gj[6];
        float ss = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            gj[j] = g[j * n + k];
            ss = fmaf(gj[j], gj[j], ss);
        }
        const float norm = sqrtf(ss);
        const bool move = norm > 0.f && isfinite(norm);
        const float scale = move ? alpha[k] / norm : 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) trial[j * n + k] = move ? p[j * n + k] - scale * gj[j] : p[j * n + k];
    }
}

__global__ void refine_accept_kernel(float* __restrict__ p, float* __restrict__ E,
                                     float* __restrict__ g, const float* __restrict__ trial,
                                     const float* __restrict__ Et, const float* __restrict__ gt,
                                     float* __restrict__ alpha, long long n, float grow,
                                     float shrink)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if (Et[k] < E[k]) {
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                p[j * n + k] = trial[j * n + k];
                g[j * n + k] = gt[j * n + k];
            }
            E[k] = Et[k];
            alpha[k] *= grow;
        } else {
            alpha[k] *= shrink;
        }
    }
}

static unsigned blocks_for(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_refine_init(float* alpha, long long n, float step0, cudaStream_t s)
{
    refine_init_kernel<<<blocks_for(n), 256, 0, s>>>(alpha, n, step0);
    return cudaGetLastError();
}

cudaError_t launch_refine_propose(const float* p, const float* g, const float* alpha,
                                  float* trial, long long n, cudaStream_t s)
{
    refine_propose_kernel<<<blocks_for(n), 256, 0, s>>>(p, g, alpha, trial, n);
    return cudaGetLastError();
}

cudaError_t launch_refine_accept(float* p, float* E, float* g, const float* trial,
                                 const float* Et, const float* gt, float* alpha, long long n,
                                 float grow, float shrink, cudaStream_t s)
{
    refine_accept_kernel<<<blocks_for(n), 256, 0, s>>>(p, E, g, trial, Et, gt, alpha, n, grow,
                                                       shrink);
    return cudaGetLastError();
}

}  // namespace bude
