// Vector kernels of the Krylov solvers: batched inner products (the Gram step
// of classical Gram-Schmidt, CGS2), multi-vector updates, norms and scalings.
// All reductions are deterministic: fixed per-thread order, fixed shuffle
// tree, and the block partials are added in block order by the last block.
// Reductions run in the precision of the vectors (FP64 vectors: FP64; FP32
// vectors: FP32) - FP64 arithmetic is a small fraction of the FP32 rate on
// this GPU, and a reduction sits on the critical path of every Krylov step.
// Results are always returned as FP64.
#include <cuda_fp16.h>
#include "ops.cuh"

namespace mg {

namespace {

// Sum a complex value over the block; result valid in thread 0.
template <typename T>
__device__ __forceinline__ C2<T> block_sum(C2<T> v, C2<T>* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    C2<T> r = mk<T>(0, 0);
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = cadd(r, sm[w]);
    }
    return r;
}

// Called by all threads after the block wrote its partials; returns true in
// every thread of the last block to arrive.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

// The last block adds the partials of all blocks: value i by warp i (mod warps),
// lanes striding over the blocks in order, then a fixed shuffle tree.  The
// partial buffer is used as C2<T>[max_blocks][RED_MAXD].
template <typename T>
__device__ __forceinline__ C2<T> warp_sum_partials(const C2<T>* partial, int i) {
    const int lane = threadIdx.x & 31;
    C2<T> acc = mk<T>(0, 0);
    for (unsigned b = lane; b < gridDim.x; b += 32) acc = cadd(acc, __ldcg(partial + (size_t)b * RED_MAXD + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void finish_reduce(double2* out, const C2<T>* partial, int nd, unsigned* ticket) {
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nd; i += nw) {
        const C2<T> acc = warp_sum_partials<T>(partial, i);
        if (lane == 0) out[i] = to_d2(acc);
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

template <typename T>
__device__ __forceinline__ void finish_reduce_real(double* out, const C2<T>* partial, unsigned* ticket) {
    __threadfence();
    if (threadIdx.x < 32) {
        const C2<T> acc = warp_sum_partials<T>(partial, 0);
        if (threadIdx.x == 0) {
            *out = (double)acc.x;
            *ticket = 0u;
        }
    }
}

constexpr int GRAM_CH = 8;

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_gram(double2* __restrict__ out, const C2<T>* __restrict__ V,
                                                      long ldv, int nd, const C2<T>* __restrict__ w, long n,
                                                      C2<T>* partial, unsigned* ticket, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> sm[RED_THREADS / 32];
    const long stride = (long)gridDim.x * blockDim.x;
    const long e0 = (long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int i0 = 0; i0 < nd; i0 += GRAM_CH) {
        C2<T> acc[GRAM_CH];
#pragma unroll
        for (int c = 0; c < GRAM_CH; ++c) acc[c] = mk<T>(0, 0);
        for (long e = e0; e < n; e += stride) {
            const C2<T> we = w[e];
#pragma unroll
            for (int c = 0; c < GRAM_CH; ++c)
                if (i0 + c < nd) acc[c] = cfmac(V[(long)(i0 + c) * ldv + e], we, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < GRAM_CH; ++c) {
            if (i0 + c < nd) {
                const C2<T> r = block_sum<T>(acc[c], sm);
                if (threadIdx.x == 0) partial[(size_t)blockIdx.x * RED_MAXD + i0 + c] = r;
            }
        }
    }
    if (last_block(ticket)) finish_reduce<T>(out, partial, nd, ticket);
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_axpy_multi(C2<T>* __restrict__ w, const C2<T>* __restrict__ V, long ldv, int nd, const int* nd_dev,
                 const double2* __restrict__ coef, double sign, int zero_first, long n, double* norm2_out,
                 C2<T>* partial, unsigned* ticket, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> cs[RED_MAXD];
    __shared__ C2<T> sm[RED_THREADS / 32];
    int cnt = nd + (nd_dev ? *nd_dev : 0);
    if (cnt > RED_MAXD) cnt = RED_MAXD;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        double2 c = coef[i];
        cs[i] = mk<T>((T)(sign * c.x), (T)(sign * c.y));
    }
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    T tacc = 0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        C2<T> a = zero_first ? mk<T>(0, 0) : w[e];
        for (int i = 0; i < cnt; ++i) a = cfma(V[(long)i * ldv + e], cs[i], a);
        w[e] = a;
        if (norm2_out) tacc += a.x * a.x + a.y * a.y;
    }
    if (norm2_out) {
        const C2<T> r = block_sum<T>(mk<T>(tacc, 0), sm);
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * RED_MAXD] = r;
        if (last_block(ticket)) finish_reduce_real<T>(norm2_out, partial, ticket);
    }
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_norm2(double* out, const C2<T>* __restrict__ v, long n,
                                                       C2<T>* partial, unsigned* ticket, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> sm[RED_THREADS / 32];
    const long stride = (long)gridDim.x * blockDim.x;
    T acc = 0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        C2<T> a = v[e];
        acc += a.x * a.x + a.y * a.y;
    }
    const C2<T> r = block_sum<T>(mk<T>(acc, 0), sm);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * RED_MAXD] = r;
    if (last_block(ticket)) finish_reduce_real<T>(out, partial, ticket);
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_redot(double* out, const C2<T>* __restrict__ x,
                                                       const C2<T>* __restrict__ y, long n, C2<T>* partial,
                                                       unsigned* ticket, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> sm[RED_THREADS / 32];
    const long stride = (long)gridDim.x * blockDim.x;
    T acc = 0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        C2<T> a = x[e], b = y[e];
        acc += a.x * b.x + a.y * b.y;
    }
    const C2<T> r = block_sum<T>(mk<T>(acc, 0), sm);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * RED_MAXD] = r;
    if (last_block(ticket)) finish_reduce_real<T>(out, partial, ticket);
}

template <typename T>
__global__ void k_scale(C2<T>* y, const C2<T>* x, const double* factor, long n, Gate g) {
    if (!gate_open(g)) return;
    const T f = (T)(*factor);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        y[e] = cscale(x[e], f);
}

template <typename Ta, typename Tb>
__global__ void k_convert(C2<Tb>* y, const C2<Ta>* x, long n, Gate g) {
    if (!gate_open(g)) return;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        C2<Ta> a = x[e];
        y[e] = mk<Tb>((Tb)a.x, (Tb)a.y);
    }
}

template <typename T>
__global__ void k_xpay(C2<T>* y, const C2<T>* x, const double* num, const double* den, long n, Gate g) {
    if (!gate_open(g)) return;
    const T a = (T)(den ? (*num / *den) : *num);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        C2<T> v = y[e], u = x[e];
        y[e] = mk<T>(u.x + a * v.x, u.y + a * v.y);
    }
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_cg_step(C2<T>* e, C2<T>* r, const C2<T>* __restrict__ p, const C2<T>* __restrict__ q, const double* rr,
              const double* pq, double* rr_new, long n, C2<T>* partial, unsigned* ticket, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> sm[RED_THREADS / 32];
    const T alpha = (T)(*rr / *pq);
    const long stride = (long)gridDim.x * blockDim.x;
    T acc = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        C2<T> pi = p[i], qi = q[i], ei = e[i], ri = r[i];
        ei.x += alpha * pi.x;
        ei.y += alpha * pi.y;
        ri.x -= alpha * qi.x;
        ri.y -= alpha * qi.y;
        e[i] = ei;
        r[i] = ri;
        acc += ri.x * ri.x + ri.y * ri.y;
    }
    const C2<T> s = block_sum<T>(mk<T>(acc, 0), sm);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * RED_MAXD] = s;
    if (last_block(ticket)) finish_reduce_real<T>(rr_new, partial, ticket);
}

inline unsigned red_blocks(long n, const RedWS& ws) {
    long b = (n + RED_THREADS - 1) / RED_THREADS;
    if (b > ws.max_blocks) b = ws.max_blocks;
    if (b < 1) b = 1;
    return (unsigned)b;
}

inline unsigned ew_blocks(long n) {
    long b = (n + 255) / 256;
    long cap = (long)sm_count() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename T> inline C2<T>* part_of(const RedWS& ws) { return reinterpret_cast<C2<T>*>(ws.partial); }

}  // namespace

template <typename T>
void launch_gram(double2* out, const C2<T>* V, long ldv, int nd, const C2<T>* w, long n, RedWS ws, Gate g,
                 cudaStream_t s) {
    if (nd <= 0) return;
    k_gram<T><<<red_blocks(n, ws), RED_THREADS, 0, s>>>(out, V, ldv, nd, w, n, part_of<T>(ws), ws.ticket, g);
    count_launch();
}

template <typename T>
void launch_axpy_multi(C2<T>* w, const C2<T>* V, long ldv, int nd, const int* nd_dev, const double2* coef,
                       double sign, bool zero_first, long n, double* norm2_out, RedWS ws, Gate g, cudaStream_t s) {
    k_axpy_multi<T><<<red_blocks(n, ws), RED_THREADS, 0, s>>>(w, V, ldv, nd, nd_dev, coef, sign, zero_first ? 1 : 0,
                                                              n, norm2_out, part_of<T>(ws), ws.ticket, g);
    count_launch();
}

template <typename T>
void launch_norm2(double* out, const C2<T>* v, long n, RedWS ws, Gate g, cudaStream_t s) {
    k_norm2<T><<<red_blocks(n, ws), RED_THREADS, 0, s>>>(out, v, n, part_of<T>(ws), ws.ticket, g);
    count_launch();
}

template <typename T>
void launch_redot(double* out, const C2<T>* x, const C2<T>* y, long n, RedWS ws, Gate g, cudaStream_t s) {
    k_redot<T><<<red_blocks(n, ws), RED_THREADS, 0, s>>>(out, x, y, n, part_of<T>(ws), ws.ticket, g);
    count_launch();
}

template <typename T>
void launch_scale(C2<T>* y, const C2<T>* x, const double* factor, long n, Gate g, cudaStream_t s) {
    k_scale<T><<<ew_blocks(n), 256, 0, s>>>(y, x, factor, n, g);
    count_launch();
}

template <typename Ta, typename Tb>
void launch_convert(C2<Tb>* y, const C2<Ta>* x, long n, Gate g, cudaStream_t s) {
    k_convert<Ta, Tb><<<ew_blocks(n), 256, 0, s>>>(y, x, n, g);
    count_launch();
}

template <typename T>
void launch_xpay(C2<T>* y, const C2<T>* x, const double* num, const double* den, long n, Gate g, cudaStream_t s) {
    k_xpay<T><<<ew_blocks(n), 256, 0, s>>>(y, x, num, den, n, g);
    count_launch();
}

template <typename T>
void launch_cg_step(C2<T>* e, C2<T>* r, const C2<T>* p, const C2<T>* q, const double* rr, const double* pq,
                    double* rr_new, long n, RedWS ws, Gate g, cudaStream_t s) {
    k_cg_step<T><<<red_blocks(n, ws), RED_THREADS, 0, s>>>(e, r, p, q, rr, pq, rr_new, n, part_of<T>(ws), ws.ticket,
                                                           g);
    count_launch();
}

#define INST(T)                                                                                                  \
    template void launch_gram<T>(double2*, const C2<T>*, long, int, const C2<T>*, long, RedWS, Gate, cudaStream_t); \
    template void launch_axpy_multi<T>(C2<T>*, const C2<T>*, long, int, const int*, const double2*, double, bool,  \
                                       long, double*, RedWS, Gate, cudaStream_t);                               \
    template void launch_norm2<T>(double*, const C2<T>*, long, RedWS, Gate, cudaStream_t);                     \
    template void launch_redot<T>(double*, const C2<T>*, const C2<T>*, long, RedWS, Gate, cudaStream_t);       \
    template void launch_scale<T>(C2<T>*, const C2<T>*, const double*, long, Gate, cudaStream_t);              \
    template void launch_xpay<T>(C2<T>*, const C2<T>*, const double*, const double*, long, Gate, cudaStream_t); \
    template void launch_cg_step<T>(C2<T>*, C2<T>*, const C2<T>*, const C2<T>*, const double*, const double*,  \
                                    double*, long, RedWS, Gate, cudaStream_t);
INST(double)
INST(float)
#undef INST
template void launch_convert<double, float>(C2<float>*, const C2<double>*, long, Gate, cudaStream_t);

// Complex FP64 -> packed FP16 pair (real part in the low half, imaginary in the
// high half), each part rounded to nearest once from FP64
__global__ void k_pack_half(unsigned* y, const double2* x, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        const unsigned re = __half_as_ushort(__double2half(v.x));
        const unsigned im = __half_as_ushort(__double2half(v.y));
        y[i] = (im << 16) | re;
    }
}
void launch_pack_half(unsigned* y, const double2* x, long n, cudaStream_t s) {
    k_pack_half<<<ew_blocks(n), 256, 0, s>>>(y, x, n);
    count_launch();
}
template void launch_convert<float, double>(C2<double>*, const C2<float>*, long, Gate, cudaStream_t);
template void launch_convert<double, double>(C2<double>*, const C2<double>*, long, Gate, cudaStream_t);
template void launch_convert<float, float>(C2<float>*, const C2<float>*, long, Gate, cudaStream_t);

}  // namespace mg
