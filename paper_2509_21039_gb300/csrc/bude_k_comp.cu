// Instantiations of the persistent pose kernel, FP32 variant kCOMP.
#include "bude_internal.h"

namespace bude {

template __global__ void pose_kernel<kCOMP, 1, false>(const Args);
template __global__ void pose_kernel<kCOMP, 2, false>(const Args);
template __global__ void pose_kernel<kCOMP, 4, false>(const Args);
template __global__ void pose_kernel<kCOMP, 8, false>(const Args);
template __global__ void pose_kernel<kCOMP, 16, false>(const Args);
template __global__ void pose_kernel<kCOMP, 1, true>(const Args);
template __global__ void pose_kernel<kCOMP, 2, true>(const Args);
template __global__ void pose_kernel<kCOMP, 4, true>(const Args);
template __global__ void pose_kernel<kCOMP, 8, true>(const Args);
template __global__ void pose_kernel<kCOMP, 2, false, true>(const Args);
template __global__ void pose_kernel<kCOMP, 4, false, true>(const Args);
template __global__ void pose_kernel<kCOMP, 8, false, true>(const Args);
template __global__ void pose_kernel<kCOMP, 16, false, true>(const Args);
template __global__ void pose_kernel<kCOMP, 2, true, true>(const Args);
template __global__ void pose_kernel<kCOMP, 4, true, true>(const Args);
template __global__ void pose_kernel<kCOMP, 8, true, true>(const Args);

const void* kernel_comp_cull(int P, bool G)
{
    if (!G) {
        switch (P) {
        case 2: return (const void*)pose_kernel<kCOMP, 2, false, true>;
        case 4: return (const void*)pose_kernel<kCOMP, 4, false, true>;
        case 8: return (const void*)pose_kernel<kCOMP, 8, false, true>;
        case 16: return (const void*)pose_kernel<kCOMP, 16, false, true>;
        }
    } else {
        switch (P) {
        case 2: return (const void*)pose_kernel<kCOMP, 2, true, true>;
        case 4: return (const void*)pose_kernel<kCOMP, 4, true, true>;
        case 8: return (const void*)pose_kernel<kCOMP, 8, true, true>;
        }
    }
    return nullptr;
}

const void* kernel_comp(int P, bool G)
{
    if (!G) {
        switch (P) {
        case 1: return (const void*)pose_kernel<kCOMP, 1, false>;
        case 2: return (const void*)pose_kernel<kCOMP, 2, false>;
        case 4: return (const void*)pose_kernel<kCOMP, 4, false>;
        case 8: return (const void*)pose_kernel<kCOMP, 8, false>;
        case 16: return (const void*)pose_kernel<kCOMP, 16, false>;
        }
    } else {
        switch (P) {
        case 1: return (const void*)pose_kernel<kCOMP, 1, true>;
        case 2: return (const void*)pose_kernel<kCOMP, 2, true>;
        case 4: return (const void*)pose_kernel<kCOMP, 4, true>;
        case 8: return (const void*)pose_kernel<kCOMP, 8, true>;
        }
    }
    return nullptr;
}

}  // namespace bude
