// The paper's memory-bound kernels (arxiv 2509.21039, Sec. 2.2, Listings 2
// and 3; metrics Eq. 1 and Eq. 2), written for GB300 as HBM calibration
// beside the compute-bound pose kernel:
//  - BabelStream copy / mul / add / triad / dot: persistent grid-stride loops
//    over 16-byte vectors with streaming (evict-first) loads and stores, four
//    vectors in flight per thread; dot reduces per warp with shuffles, per
//    CTA in shared memory and over CTAs in a fixed order (FP64 partials).
//  - Seven-point stencil: each thread keeps a column of CH + 2 values along
//    the slowest index in registers and reads the j/k neighbours through the
//    read-only path (L1 hits inside the CTA's tile); no barriers, so many
//    independent loads are in flight.
#include <algorithm>

#include "bude_internal.h"

namespace bude {

template <typename T> struct Vec;
template <> struct Vec<float> { typedef float4 V; static constexpr int N = 4; };
template <> struct Vec<double> { typedef double2 V; static constexpr int N = 2; };

__device__ __forceinline__ float4 vmul(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ double2 vmul(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float4 vadd(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 vfma(float s, float4 c, float4 b)
{
    return make_float4(fmaf(s, c.x, b.x), fmaf(s, c.y, b.y), fmaf(s, c.z, b.z), fmaf(s, c.w, b.w));
}
__device__ __forceinline__ double2 vfma(double s, double2 c, double2 b)
{
    return make_double2(fma(s, c.x, b.x), fma(s, c.y, b.y));
}
// Per-thread dot accumulators.  FP32: a Neumaier-compensated FP32 sum (FP64
// arithmetic is slow on this GPU and would bound the kernel); FP64: FMAs.
struct DotAcc32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
struct DotAcc64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
__device__ __forceinline__ void vdot(DotAcc32& acc, float4 a, float4 b)
{
    acc.add(fmaf(a.y, b.y, a.x * b.x));
    acc.add(fmaf(a.w, b.w, a.z * b.z));
}
__device__ __forceinline__ void vdot(DotAcc64& acc, double2 a, double2 b)
{
    acc.s = fma(a.x, b.x, acc.s);
    acc.s = fma(a.y, b.y, acc.s);
}
template <typename T> struct DotAcc { typedef DotAcc32 A; };
template <> struct DotAcc<double> { typedef DotAcc64 A; };

enum StreamOp { kCopy = 0, kMul = 1, kAdd = 2, kTriad = 3, kDot = 4 };
constexpr int kUnroll = 4;

// One element-wise op over nv vectors (vector part) plus a scalar tail.
template <typename T, int OP>
__global__ void stream_kernel(T* __restrict__ a, T* __restrict__ b, T* __restrict__ c, T s,
                              long long n, double* __restrict__ partial)
{
    typedef typename Vec<T>::V V;
    constexpr int NV = Vec<T>::N;
    const long long nv = n / NV;
    V* av = reinterpret_cast<V*>(a);
    V* bv = reinterpret_cast<V*>(b);
    V* cv = reinterpret_cast<V*>(c);
    const long long stride = (long long)gridDim.x * blockDim.x;
    typename DotAcc<T>::A acc;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kUnroll - 1) * stride < nv; i += kUnroll * stride) {
        V x[kUnroll], y[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long j = i + u * stride;
            if (OP == kCopy || OP == kAdd || OP == kDot) x[u] = __ldcs(av + j);
            if (OP == kMul || OP == kTriad) x[u] = __ldcs(cv + j);
            if (OP == kAdd || OP == kTriad || OP == kDot) y[u] = __ldcs(bv + j);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long j = i + u * stride;
            if (OP == kCopy) __stcs(cv + j, x[u]);
            if (OP == kMul) __stcs(bv + j, vmul(s, x[u]));
            if (OP == kAdd) __stcs(cv + j, vadd(x[u], y[u]));
            if (OP == kTriad) __stcs(av + j, vfma(s, x[u], y[u]));
            if (OP == kDot) vdot(acc, x[u], y[u]);
        }
    }
    for (; i < nv; i += stride) {
        if (OP == kCopy) __stcs(cv + i, __ldcs(av + i));
        if (OP == kMul) __stcs(bv + i, vmul(s, __ldcs(cv + i)));
        if (OP == kAdd) __stcs(cv + i, vadd(__ldcs(av + i), __ldcs(bv + i)));
        if (OP == kTriad) __stcs(av + i, vfma(s, __ldcs(cv + i), __ldcs(bv + i)));
        if (OP == kDot) vdot(acc, __ldcs(av + i), __ldcs(bv + i));
    }
    // scalar tail (n not a multiple of the vector width)
    const long long t0 = nv * NV;
    for (long long e = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        if (OP == kCopy) c[e] = a[e];
        if (OP == kMul) b[e] = s * c[e];
        if (OP == kAdd) c[e] = a[e] + b[e];
        if (OP == kTriad) a[e] = b[e] + s * c[e];
        if (OP == kDot) acc.add(a[e] * b[e]);
    }
    if (OP == kDot) {
        __shared__ double s_w[32];
        double v = acc.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_w[w];
            partial[blockIdx.x] = v;
        }
    }
}

// Sum of the per-CTA partials by one CTA of 1024 threads: each thread adds
// the partials i = tid, tid + 1024, ... in order, then a butterfly per warp
// and the 32 warp sums in warp order.  The order is fixed, so the result is
// deterministic; a serial loop here cost tens of microseconds at 2^25.
__global__ void __launch_bounds__(1024) dot_finish_kernel(const double* __restrict__ partial, int n,
                                                          double* __restrict__ out)
{
    __shared__ double s_w[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) *out = w;
    }
}

// f[i,j,k] on interior points; index i*ny*nz + j*nz + k (k fastest).  Each
// thread owns one (j, k) column for CH consecutive planes of chunk
// blockIdx.z: its column values u[i0-1 .. i0+CH] and the j/k neighbours of
// its CH points are all loaded before any arithmetic, with the plane index
// clamped into the array instead of a guard, so that every load of the
// thread is independent and in flight at once; the stores alone are
// predicated.  The j/k neighbours come through the read-only path, where the
// CTA's tile makes most of them L1 hits.  No barriers.
template <typename T, int TX, int TY, int CH>
__global__ void __launch_bounds__(TX * TY) laplacian_kernel(const T* __restrict__ u,
                                                            T* __restrict__ f, int nx, int ny,
                                                            int nz, T cx, T cy, T cz, T c0)
{
    const int k = blockIdx.x * TX + threadIdx.x + 1, j = blockIdx.y * TY + threadIdx.y + 1;
    const int i0 = 1 + blockIdx.z * CH;
    const int i1 = min(nx - 1, i0 + CH);
    if (k >= nz - 1 || j >= ny - 1 || i0 >= i1) return;
    const size_t plane = (size_t)ny * nz;
    const size_t col = (size_t)j * nz + k;
    T c[CH + 2], yn[CH], yp[CH], zn[CH], zp[CH];
#pragma unroll
    for (int q = 0; q < CH + 2; ++q) {
        const int i = min(i0 - 1 + q, nx - 1);
        c[q] = __ldg(u + (size_t)i * plane + col);
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        const size_t o = (size_t)min(i0 + q, nx - 1) * plane + col;
        yn[q] = __ldg(u + o - nz);
        yp[q] = __ldg(u + o + nz);
        zn[q] = __ldg(u + o - 1);
        zp[q] = __ldg(u + o + 1);
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        const int i = i0 + q;
        if (i < i1)
            f[(size_t)i * plane + col] = c[q + 1] * c0 + (c[q] + c[q + 2]) * cx +
                                         (yn[q] + yp[q]) * cy + (zn[q] + zp[q]) * cz;
    }
}

// Partial sums of dot: one slot per CTA of the launch, shared by all calls
// (the library's fixed device array; calls must not overlap on the GPU).
constexpr int kMaxStreamCtas = 4096;
static __device__ double g_dot_partial[kMaxStreamCtas];

}  // namespace bude

using namespace bude;

namespace {

template <typename T>
cudaError_t stream_launch(int op, T* a, T* b, T* c, T s, long long n, double* dot_out,
                          cudaStream_t st, int* launches)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    long long want = (n / Vec<T>::N + threads * kUnroll - 1) / (threads * kUnroll);
    long long grid = std::max(1ll, std::min<long long>(want, (long long)sms * 8));
    grid = std::min<long long>(grid, kMaxStreamCtas);
    double* partial = nullptr;
    if (op == kDot) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_partial);
        if (e != cudaSuccess) return e;
        partial = static_cast<double*>(p);
    }
    switch (op) {
    case kCopy: stream_kernel<T, kCopy><<<(unsigned)grid, threads, 0, st>>>(a, b, c, s, n, partial); break;
    case kMul: stream_kernel<T, kMul><<<(unsigned)grid, threads, 0, st>>>(a, b, c, s, n, partial); break;
    case kAdd: stream_kernel<T, kAdd><<<(unsigned)grid, threads, 0, st>>>(a, b, c, s, n, partial); break;
    case kTriad: stream_kernel<T, kTriad><<<(unsigned)grid, threads, 0, st>>>(a, b, c, s, n, partial); break;
    case kDot: stream_kernel<T, kDot><<<(unsigned)grid, threads, 0, st>>>(a, b, c, s, n, partial); break;
    }
    cudaError_t e = cudaGetLastError();
    *launches = 1;
    if (e == cudaSuccess && op == kDot) {
        dot_finish_kernel<<<1, 1024, 0, st>>>(partial, (int)grid, dot_out);
        e = cudaGetLastError();
        *launches = 2;
    }
    return e;
}

template <typename T>
cudaError_t laplacian_launch(const T* u, T* f, int nx, int ny, int nz, T cx, T cy, T cz, T c0,
                             cudaStream_t st)
{
    constexpr int TX = 64, TY = 4, CH = 8;
    dim3 grid((unsigned)((nz - 2 + TX - 1) / TX), (unsigned)((ny - 2 + TY - 1) / TY),
              (unsigned)((nx - 2 + CH - 1) / CH));
    laplacian_kernel<T, TX, TY, CH><<<grid, dim3(TX, TY), 0, st>>>(u, f, nx, ny, nz, cx, cy, cz, c0);
    return cudaGetLastError();
}

}  // namespace

extern "C" BUDE_API int bude_stream(int32_t op, int32_t dtype, void* a, void* b, void* c,
                                    double scalar, int64_t n, double* dot_result, void* stream)
{
    Range range_("bude_stream");
    if (op < 0 || op > 4 || (dtype != 0 && dtype != 1) || n < 0) return BUDE_ERR_INVALID_ARG;
    if (n == 0) {
        if (op == kDot && dot_result)
            return cudaMemsetAsync(dot_result, 0, sizeof(double), (cudaStream_t)stream) == cudaSuccess
                       ? BUDE_OK : BUDE_ERR_CUDA;
        return BUDE_OK;
    }
    const bool need_a = op != kMul, need_b = op != kCopy, need_c = op != kDot;
    if ((need_a && !a) || (need_b && !b) || (need_c && !c) || (op == kDot && !dot_result))
        return BUDE_ERR_INVALID_ARG;
    // 16-byte vectors need 16-byte aligned arrays
    const uintptr_t mis = ((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u;
    if (mis) return BUDE_ERR_INVALID_ARG;
    int launches = 0;
    cudaError_t e;
    if (dtype == 0)
        e = stream_launch<float>(op, (float*)a, (float*)b, (float*)c, (float)scalar, n, dot_result,
                                 (cudaStream_t)stream, &launches);
    else
        e = stream_launch<double>(op, (double*)a, (double*)b, (double*)c, scalar, n, dot_result,
                                  (cudaStream_t)stream, &launches);
    return e == cudaSuccess ? BUDE_OK : BUDE_ERR_CUDA;
}

extern "C" BUDE_API int bude_laplacian(int32_t dtype, const void* u, void* f, int32_t nx,
                                       int32_t ny, int32_t nz, double invhx2, double invhy2,
                                       double invhz2, double invhxyz2, void* stream)
{
    Range range_("bude_laplacian");
    if ((dtype != 0 && dtype != 1) || nx < 0 || ny < 0 || nz < 0) return BUDE_ERR_INVALID_ARG;
    if (nx < 3 || ny < 3 || nz < 3) return BUDE_OK;  // no interior points
    if (!u || !f || u == f) return BUDE_ERR_INVALID_ARG;
    if ((long long)(ny - 2 + 7) / 8 > 65535 || (long long)(nx - 2 + 7) / 8 > 65535)
        return BUDE_ERR_UNSUPPORTED;
    cudaError_t e;
    if (dtype == 0)
        e = laplacian_launch<float>((const float*)u, (float*)f, nx, ny, nz, (float)invhx2,
                                    (float)invhy2, (float)invhz2, (float)invhxyz2,
                                    (cudaStream_t)stream);
    else
        e = laplacian_launch<double>((const double*)u, (double*)f, nx, ny, nz, invhx2, invhy2,
                                     invhz2, invhxyz2, (cudaStream_t)stream);
    return e == cudaSuccess ? BUDE_OK : BUDE_ERR_CUDA;
}
