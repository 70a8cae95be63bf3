// dcsd_selftest_conversions: checks the integer-unit FP64 <-> FP32
// conversions (f32_to_f64, f64_to_f32 in common.h) against the hardware
// conversions on the device they will run on.
#include "common.h"

namespace {
using dcsd::f32_to_f64;
using dcsd::f64_to_f32;

// counter-based 64-bit mixer (splitmix64 finaliser) for the test patterns
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool same_f32(float a, float b) {
    return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}
__device__ __forceinline__ bool same_f64(double a, double b) {
    return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}

// every binary32 bit pattern -> binary64
__global__ void k_check_f32_to_f64(unsigned long long* bad) {
    unsigned long long nbad = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (1ull << 32);
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float x = __uint_as_float((unsigned)i);
        if (!same_f64(f32_to_f64(x), (double)x)) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
}

// binary64 patterns: every biased exponent, random sign and fraction, with
// the 29 fraction bits dropped by the rounding forced to 0, to the tie, to
// the tie +- 1 and to their maximum in turn
__global__ void k_check_f64_to_f32(unsigned long long n, unsigned long long* bad) {
    unsigned long long nbad = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r = mix64(i);
        const unsigned long long e = (i >> 3) % 2048ull;
        unsigned long long frac = r & 0xFFFFFFFFFFFFFull;
        const unsigned long long low = frac & 0x1FFFFFFFull;
        const unsigned long long hiF = frac & ~0x1FFFFFFFull;
        switch (i & 7ull) {
            case 0: frac = hiF; break;
            case 1: frac = hiF | 0x10000000ull; break;
            case 2: frac = hiF | 0x0FFFFFFFull; break;
            case 3: frac = hiF | 0x10000001ull; break;
            case 4: frac = hiF | 0x1FFFFFFFull; break;
            case 5: frac = 0xFFFFFFFFFFFFFull; break;
            default: frac = hiF | low; break;
        }
        const unsigned long long bits = (r & 0x8000000000000000ull) | (e << 52) | frac;
        const double x = __longlong_as_double((long long)bits);
        if (!same_f32(f64_to_f32(x), (float)x)) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
}

}  // namespace

extern "C" dcsd_status dcsd_selftest_conversions(void* stream, long long* mismatches) {
    if (!mismatches) return DCSD_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return DCSD_ERR_NO_DEVICE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* d = nullptr;
    if (cudaMalloc((void**)&d, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return DCSD_ERR_OOM;
    }
    dcsd_status status = DCSD_OK;
    unsigned long long h = 0;
    if (cudaMemsetAsync(d, 0, sizeof(*d), st) != cudaSuccess) status = DCSD_ERR_CUDA;
    if (status == DCSD_OK) {
        k_check_f32_to_f64<<<4096, 256, 0, st>>>(d);
        k_check_f64_to_f32<<<4096, 256, 0, st>>>(1ull << 28, d);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            status = DCSD_ERR_CUDA;
    }
    cudaFree(d);
    if (status == DCSD_OK) *mismatches = (long long)h;
    return status;
}
