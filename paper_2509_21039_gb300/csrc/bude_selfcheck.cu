// Self-check of the branch-free square root used by the IEEE energy kernels:
// every float x in [2^-100, 2^128) (the range the kernels feed it) is
// compared bit for bit with the correctly rounded sqrt.rn.
#include "bude_internal.h"

namespace bude {

__global__ void sqrt_selfcheck_kernel(unsigned long long lo, unsigned long long hi,
                                      unsigned long long* mismatches, unsigned* first_bad)
{
    unsigned long long bad = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long b = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         b < hi; b += stride) {
        const float x = __uint_as_float((unsigned)b);
        if (__float_as_uint(sqrt_rn_fma(x)) != __float_as_uint(__fsqrt_rn(x))) {
            ++bad;
            atomicMin(first_bad, (unsigned)b);
        }
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace bude

extern "C" BUDE_API int bude_selfcheck_sqrt(uint64_t* mismatches, uint32_t* first_bad,
                                            void* stream)
{
    bude::Range range_("bude_selfcheck_sqrt");
    if (!mismatches) return BUDE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    struct R { unsigned long long n; unsigned first; unsigned pad; };
    R* d = nullptr;
    if (bude::dev_alloc((void**)&d, sizeof(R)) != cudaSuccess) return BUDE_ERR_OOM;
    R h{0ull, 0xffffffffu, 0u};
    cudaError_t e = cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        bude::sqrt_selfcheck_kernel<<<152 * 8, 256, 0, s>>>(0x0d800000ull, 0x7f800000ull, &d->n,
                                                            &d->first);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return BUDE_ERR_CUDA;
    *mismatches = h.n;
    if (first_bad) *first_bad = h.first;
    return BUDE_OK;
}
