// Shared device helpers of the solver library: complex arithmetic on
// interleaved (re, im) pairs, error reporting, launch geometry.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/mg.h"

namespace mg {

// ---------------------------------------------------------------- complex ----
template <typename T> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename T> using C2 = typename cplx_of<T>::type;

template <typename T> __host__ __device__ __forceinline__ C2<T> mk(T r, T i) {
    C2<T> z;
    z.x = r;
    z.y = i;
    return z;
}
template <typename Z> __host__ __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z cneg(Z a) { a.x = -a.x; a.y = -a.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z conj_(Z a) { a.y = -a.y; return a; }
template <typename Z, typename R> __host__ __device__ __forceinline__ Z cscale(Z a, R s) { a.x *= s; a.y *= s; return a; }
// a * b
template <typename Z> __host__ __device__ __forceinline__ Z cmul(Z a, Z b) {
    Z c;
    c.x = a.x * b.x - a.y * b.y;
    c.y = a.x * b.y + a.y * b.x;
    return c;
}
// conj(a) * b
template <typename Z> __host__ __device__ __forceinline__ Z cmulc(Z a, Z b) {
    Z c;
    c.x = a.x * b.x + a.y * b.y;
    c.y = a.x * b.y - a.y * b.x;
    return c;
}
// acc + a * b
template <typename Z> __host__ __device__ __forceinline__ Z cfma(Z a, Z b, Z acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
template <typename Z> __host__ __device__ __forceinline__ Z cfmac(Z a, Z b, Z acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
// i * a
template <typename Z> __host__ __device__ __forceinline__ Z cmuli(Z a) { Z c; c.x = -a.y; c.y = a.x; return c; }
template <typename Z> __host__ __device__ __forceinline__ double cabs2(Z a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T> __host__ __device__ __forceinline__ C2<T> from_d2(double2 a) {
    return mk<T>((T)a.x, (T)a.y);
}

// ------------------------------------------------------------------ errors ---
void set_error(const char* fmt, ...);

#define MG_CUDA_TRY(expr)                                                                     \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            ::mg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                            __LINE__);                                                        \
            return MG_ECUDA;                                                                  \
        }                                                                                     \
    } while (0)

#define MG_TRY(expr)                      \
    do {                                  \
        mg_status _s = (expr);            \
        if (_s != MG_OK) return _s;       \
    } while (0)

// check the last launch
#define MG_LAUNCH_CHECK() MG_CUDA_TRY(cudaGetLastError())

inline unsigned nblocks(long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// number of SMs of the current device (cached per process for device 0..15)
int sm_count();

// process-wide count of kernel launches made by this library
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace mg
