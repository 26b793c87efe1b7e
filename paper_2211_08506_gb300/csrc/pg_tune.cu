// Small device reductions used by the autotuner to check each launch candidate against
// the first one: an order-independent hash of a buffer's bits (bitwise equality) and
// max|a-b| / max|b| over two grids of the same dtype (tolerance check).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pg_internal.h"

namespace pgi {

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    // SplitMix64 finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
    // generators", OOPSLA 2014).
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void hash_kernel(const uint4 *words4, size_t n4, const unsigned *tail, size_t n_tail,
                            unsigned long long *out)
{
    unsigned long long s = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint4 w = words4[i];
        const unsigned long long base = (unsigned long long)(4 * i) << 32;
        s += mix64(base ^ w.x) + mix64((base + (1ull << 32)) ^ w.y) +
             mix64((base + (2ull << 32)) ^ w.z) + mix64((base + (3ull << 32)) ^ w.w);
    }
    if (blockIdx.x == 0)
        for (size_t i = threadIdx.x; i < n_tail; i += blockDim.x)
            s += mix64(((unsigned long long)(4 * n4 + i) << 32) ^ tail[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ unsigned long long part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(out, t);
    }
}

template <typename T>
__device__ __forceinline__ float as_f(T v);
template <>
__device__ __forceinline__ float as_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float as_f<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float as_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void compare_kernel(const T *a, const T *b, size_t n, float *out2)
{
    float md = 0.0f, mb = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float x = as_f<T>(a[i]), y = as_f<T>(b[i]);
        const float d = fabsf(x - y);
        md = fmaxf(md, d != d ? INFINITY : d);  // NaN counts as a mismatch
        mb = fmaxf(mb, fabsf(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<int *>(out2), __float_as_int(md));
        atomicMax(reinterpret_cast<int *>(out2 + 1), __float_as_int(mb));
    }
}

}  // namespace

cudaError_t buffer_hash(const void *buf, size_t bytes, unsigned long long *d_out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const size_t n = bytes / 4;
    if (n == 0) return cudaSuccess;
    // 16-byte words where the buffer is 16-byte aligned, the remainder word by word.
    const bool aligned = ((uintptr_t)buf % 16) == 0;
    const size_t n4 = aligned ? n / 4 : 0;
    const unsigned *tail = reinterpret_cast<const unsigned *>(buf) + 4 * n4;
    hash_kernel<<<2048, 256, 0, s>>>(reinterpret_cast<const uint4 *>(buf), n4, tail, n - 4 * n4,
                                     d_out);
    return cudaGetLastError();
}

cudaError_t buffer_compare(const void *a, const void *b, size_t n, int dtype, float *d_out2,
                           cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_out2, 0, 2 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    if (dtype == PG_F32)
        compare_kernel<float><<<512, 256, 0, s>>>((const float *)a, (const float *)b, n, d_out2);
    else if (dtype == PG_F16)
        compare_kernel<__half><<<512, 256, 0, s>>>((const __half *)a, (const __half *)b, n, d_out2);
    else
        compare_kernel<__nv_bfloat16><<<512, 256, 0, s>>>((const __nv_bfloat16 *)a,
                                                          (const __nv_bfloat16 *)b, n, d_out2);
    return cudaGetLastError();
}

}  // namespace pgi
