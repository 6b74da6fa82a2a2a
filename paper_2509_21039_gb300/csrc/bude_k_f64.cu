// Instantiations of the persistent pose kernel, FP64 variant.
#include "bude_internal.h"

namespace bude {

template __global__ void pose_kernel<kF64, 1, false>(const Args);
template __global__ void pose_kernel<kF64, 2, false>(const Args);
template __global__ void pose_kernel<kF64, 4, false>(const Args);
template __global__ void pose_kernel<kF64, 1, true>(const Args);
template __global__ void pose_kernel<kF64, 2, true>(const Args);
template __global__ void pose_kernel<kF64, 4, true>(const Args);

const void* kernel_f64(int P, bool G)
{
    switch (P) {
    case 1: return G ? (const void*)pose_kernel<kF64, 1, true> : (const void*)pose_kernel<kF64, 1, false>;
    case 2: return G ? (const void*)pose_kernel<kF64, 2, true> : (const void*)pose_kernel<kF64, 2, false>;
    case 4: return G ? (const void*)pose_kernel<kF64, 4, true> : (const void*)pose_kernel<kF64, 4, false>;
    }
    return nullptr;
}

}  // namespace bude
