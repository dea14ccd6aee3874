// Kernels of the lockstep multi-right-hand-side solve (batch.cuh):
//  * batched inner products, multi-vector updates, norms and scalings, one
//    launch for a whole block of right-hand sides, each right-hand side reduced
//    deterministically (fixed per-thread order, fixed shuffle tree, the chunk
//    partials added in chunk order by the last chunk of that right-hand side);
//  * the 24-dof block stencil of the intermediate and coarsest grids
//    (D^ = P^+ D P, Section 2) for a block of right-hand sides on tensor cores.
//
// Tensor-core block products.  For one site s and one direction d the 5-point
// stencil multiplies a complex 24 x 24 block A by the complex 24-vectors of
// eight right-hand sides at the neighbour: a complex (24 x 24)(24 x 8) product.
// With the real embedding that keeps real and imaginary parts interleaved,
//   [re y_a]   [re A_ac  -im A_ac] [re x_c]
//   [im y_a] = [im A_ac   re A_ac] [im x_c],
// the product is a real (48 x 48)(48 x 8) one, i.e. 3 x 3 tiles of
// mma.sync.m16n8k16 (BF16 or FP16 inputs, FP32 accumulation), and the vector's
// natural layout (re, im, re, im, ...) is exactly the K order of the B operand.
// The operator is stored once per apply-format as complex 16-bit pairs in the
// order the A fragments are loaded (one 16-byte load per thread per tile); the
// embedding (a sign flip or a half swap) is formed in registers.  The FP32
// vectors are split into x = hi + lo, both rounded to the 16-bit format, and
// multiplied twice, so the product carries the operator's rounding only.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch.cuh"

namespace mg {

namespace {

// ------------------------------------------------------------ batched BLAS --

template <typename T>
__device__ __forceinline__ C2<T> bblock_sum(C2<T> v, C2<T>* sm) {
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
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = cadd(r, sm[w]);
    return r;
}

// true in every thread of the last chunk block of right-hand side r
__device__ __forceinline__ bool blast_chunk(unsigned* ticket) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    return am_last;
}

// sum over the chunks of value i of right-hand side r, in chunk order, by one warp
template <typename T>
__device__ __forceinline__ C2<T> bsum_chunks(const C2<T>* part_r, int i) {
    const int lane = threadIdx.x & 31;
    C2<T> acc = mk<T>(0, 0);
    for (unsigned c = lane; c < gridDim.x; c += 32) acc = cadd(acc, __ldcg(part_r + (size_t)c * RED_MAXD + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    return acc;
}

constexpr int BT = 256;      // threads of the batched BLAS kernels
constexpr int BGRAM_CH = 8;  // inner products per pass over the vector

template <typename T>
__global__ void __launch_bounds__(BT) k_bgram(double2* __restrict__ out, long os, const C2<T>* __restrict__ V,
                                              long ldv, long vr, int nd, const int* ndd, long nds,
                                              const C2<T>* __restrict__ w, long wr, long n, C2<T>* partial,
                                              int max_chunks, unsigned* ticket, Gate g) {
    const int r = blockIdx.y;
    if (!gate_open(g, r)) return;
    __shared__ C2<T> sm[BT / 32];
    int cnt = nd + (ndd ? ndd[r * nds] : 0);
    if (cnt > RED_MAXD) cnt = RED_MAXD;
    const C2<T>* Vr = V + r * vr;
    const C2<T>* wv = w + r * wr;
    C2<T>* part_r = partial + (size_t)r * max_chunks * RED_MAXD;
    const long stride = (long)gridDim.x * BT;
    const long e0 = (long)blockIdx.x * BT + threadIdx.x;
    for (int i0 = 0; i0 < cnt; i0 += BGRAM_CH) {
        C2<T> acc[BGRAM_CH];
#pragma unroll
        for (int c = 0; c < BGRAM_CH; ++c) acc[c] = mk<T>(0, 0);
        for (long e = e0; e < n; e += stride) {
            const C2<T> we = wv[e];
#pragma unroll
            for (int c = 0; c < BGRAM_CH; ++c)
                if (i0 + c < cnt) acc[c] = cfmac(Vr[(long)(i0 + c) * ldv + e], we, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < BGRAM_CH; ++c)
            if (i0 + c < cnt) {
                const C2<T> v = bblock_sum<T>(acc[c], sm);
                if (threadIdx.x == 0) part_r[(size_t)blockIdx.x * RED_MAXD + i0 + c] = v;
            }
    }
    if (blast_chunk(ticket + r)) {
        __threadfence();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int i = warp; i < cnt; i += BT / 32) {
            const C2<T> v = bsum_chunks<T>(part_r, i);
            if (lane == 0) out[r * os + i] = to_d2(v);
        }
        if (threadIdx.x == 0) ticket[r] = 0u;
    }
}

template <typename T>
__global__ void __launch_bounds__(BT) k_baxpy(C2<T>* w, long wr, const C2<T>* __restrict__ V, long ldv, long vr,
                                              int nd, const int* ndd, long nds, const double2* __restrict__ coef,
                                              long cs, double sign, int zero_first, long n, double* norm2, long n2s,
                                              C2<T>* partial, int max_chunks, unsigned* ticket, Gate g) {
    const int r = blockIdx.y;
    if (!gate_open(g, r)) return;
    __shared__ C2<T> cf[RED_MAXD];
    __shared__ C2<T> sm[BT / 32];
    int cnt = nd + (ndd ? ndd[r * nds] : 0);
    if (cnt > RED_MAXD) cnt = RED_MAXD;
    for (int i = threadIdx.x; i < cnt; i += BT) {
        const double2 c = coef[r * cs + i];
        cf[i] = mk<T>((T)(sign * c.x), (T)(sign * c.y));
    }
    __syncthreads();
    const C2<T>* Vr = V + r * vr;
    C2<T>* wv = w + r * wr;
    const long stride = (long)gridDim.x * BT;
    T tacc = 0;
    for (long e = (long)blockIdx.x * BT + threadIdx.x; e < n; e += stride) {
        C2<T> a = zero_first ? mk<T>(0, 0) : wv[e];
        for (int i = 0; i < cnt; ++i) a = cfma(Vr[(long)i * ldv + e], cf[i], a);
        wv[e] = a;
        if (norm2) tacc += a.x * a.x + a.y * a.y;
    }
    if (norm2) {
        C2<T>* part_r = partial + (size_t)r * max_chunks * RED_MAXD;
        const C2<T> v = bblock_sum<T>(mk<T>(tacc, 0), sm);
        if (threadIdx.x == 0) part_r[(size_t)blockIdx.x * RED_MAXD] = v;
        if (blast_chunk(ticket + r)) {
            __threadfence();
            if (threadIdx.x < 32) {
                const C2<T> t = bsum_chunks<T>(part_r, 0);
                if (threadIdx.x == 0) {
                    norm2[r * n2s] = (double)t.x;
                    ticket[r] = 0u;
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(BT) k_bnorm2(double* out, long os, const C2<T>* __restrict__ v, long vr, long n,
                                               C2<T>* partial, int max_chunks, unsigned* ticket, Gate g) {
    const int r = blockIdx.y;
    if (!gate_open(g, r)) return;
    __shared__ C2<T> sm[BT / 32];
    const C2<T>* vv = v + r * vr;
    const long stride = (long)gridDim.x * BT;
    T acc = 0;
    for (long e = (long)blockIdx.x * BT + threadIdx.x; e < n; e += stride) {
        const C2<T> a = vv[e];
        acc += a.x * a.x + a.y * a.y;
    }
    C2<T>* part_r = partial + (size_t)r * max_chunks * RED_MAXD;
    const C2<T> s = bblock_sum<T>(mk<T>(acc, 0), sm);
    if (threadIdx.x == 0) part_r[(size_t)blockIdx.x * RED_MAXD] = s;
    if (blast_chunk(ticket + r)) {
        __threadfence();
        if (threadIdx.x < 32) {
            const C2<T> t = bsum_chunks<T>(part_r, 0);
            if (threadIdx.x == 0) {
                out[r * os] = (double)t.x;
                ticket[r] = 0u;
            }
        }
    }
}

template <typename T>
__global__ void k_bscale(C2<T>* y, long yr, const C2<T>* x, long xr, const double* f, long fs, long n, Gate g) {
    const int r = blockIdx.y;
    if (!gate_open(g, r)) return;
    const T fv = (T)f[r * fs];
    C2<T>* yy = y + r * yr;
    const C2<T>* xx = x + r * xr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        yy[e] = cscale(xx[e], fv);
}

template <typename Ta, typename Tb>
__global__ void k_bconvert(C2<Tb>* y, long yr, const C2<Ta>* x, long xr, long n) {
    const int r = blockIdx.y;
    C2<Tb>* yy = y + r * yr;
    const C2<Ta>* xx = x + r * xr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const C2<Ta> a = xx[e];
        yy[e] = mk<Tb>((Tb)a.x, (Tb)a.y);
    }
}

inline int chunks_for(long n, const BRed& red) {
    long c = (n + BT * 4 - 1) / (BT * 4);
    if (c > red.max_chunks) c = red.max_chunks;
    if (c < 1) c = 1;
    return (int)c;
}
inline unsigned ew_chunks(long n) {
    long c = (n + 1023) / 1024;
    if (c > 64) c = 64;
    if (c < 1) c = 1;
    return (unsigned)c;
}

// ------------------------------------------------------ tensor-core stencil --

constexpr int NDOF = 24;
constexpr int TILE_WORDS = 64;                    // one 8 x 8 complex tile
constexpr int SITE_WORDS = 5 * 9 * TILE_WORDS;    // 5 directions x 3 x 3 tiles

template <bool F16>
__device__ __forceinline__ unsigned pack16(float re, float im) {
    if constexpr (F16) {
        const __half2 h = __floats2half2_rn(re, im);  // .x (low) = re, .y (high) = im
        return *reinterpret_cast<const unsigned*>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        return *reinterpret_cast<const unsigned*>(&h);
    }
}
template <bool F16>
__device__ __forceinline__ float2 unpack16(unsigned u) {
    if constexpr (F16) {
        const __half2 h = *reinterpret_cast<const __half2*>(&u);
        return __half22float2(h);
    } else {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&u);
        return __bfloat1622float2(h);
    }
}

template <bool F16>
__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    if constexpr (F16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// A fragment word of the real embedding from a complex pair (re low, im high):
// rows of real parts take (re, -im), rows of imaginary parts (im, re)
__device__ __forceinline__ unsigned embed(unsigned w, int p) {
    return p ? __byte_perm(w, 0u, 0x1032) : (w ^ 0x80000000u);
}

// neighbour site in direction d (self, +x, -x, +t, -t), periodic; 32-bit index
// arithmetic (a coarse grid has far fewer than 2^31 sites)
__device__ __forceinline__ int nbr_of(int s, int d, int Nx, int Nt) {
    const int t = s / Nx, xx = s - t * Nx;
    switch (d) {
        case 0: return s;
        case 1: return (xx + 1 == Nx) ? s - xx : s + 1;
        case 2: return (xx == 0) ? s + Nx - 1 : s - 1;
        case 3: return (t + 1 == Nt) ? xx : s + Nx;
        default: return (t == 0) ? s + Nx * (Nt - 1) : s - Nx;
    }
}

// FP64 -> BF16 rounded once to nearest-even: the FP64 significand is rounded at
// BF16's 8 significant bits (bit 45 of the FP64 word is the last kept one), after
// which the value converts to FP32 and to BF16 exactly (operator entries are far
// inside BF16's exponent range)
__device__ __forceinline__ unsigned short bf16_rn(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    u += 0x00000FFFFFFFFFFFull + ((u >> 45) & 1ull);
    u &= 0xFFFFE00000000000ull;
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)__longlong_as_double((long long)u)));
}

// Fragment order of a tile (output rows 8 mt + a, input columns 8 kt + c):
// word 4 (4 a0 + t) + e holds entry (a0 + 4 (e & 1), t + 4 (e >> 1)), so the
// thread of group g (rows g, g + 8 of the real tile) and lane-in-group t loads
// the four entries of its A fragment as one 16-byte vector at 4 (g / 2) + t.
template <bool F16>
__global__ void k_pack_frag(unsigned* out, const double2* __restrict__ A, long nsite) {
    const long total = nsite * SITE_WORDS;
    for (long w = (long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long)gridDim.x * blockDim.x) {
        const long tile = w / TILE_WORDS;
        const int q = (int)(w - tile * TILE_WORDS);
        const int e = q & 3, t = (q >> 2) & 3, a0 = q >> 4;
        const long sd = tile / 9;  // site * 5 + direction
        const int mk_ = (int)(tile - sd * 9), mt = mk_ / 3, kt = mk_ - 3 * mt;
        const int row = 8 * mt + a0 + 4 * (e & 1), col = 8 * kt + t + 4 * (e >> 1);
        const double2 v = A[(sd * NDOF + col) * NDOF + row];  // column-major block: entry (row, col)
        unsigned re, im;
        if constexpr (F16) {
            re = __half_as_ushort(__double2half(v.x));
            im = __half_as_ushort(__double2half(v.y));
        } else {
            re = bf16_rn(v.x);
            im = bf16_rn(v.y);
        }
        out[w] = (im << 16) | re;
    }
}

// One CTA per group of G = max(1, 8 / ntiles) sites, one warp per (site, tile of
// 8 right-hand sides).  The CTA stages the operator of its sites into shared
// memory once (cp.async, 11.5 KB a site), so every tile of a site reads the same
// copy; each warp issues all its neighbour-vector loads before it waits, so a
// CTA pays one round of memory latency.
template <bool F16, bool RES>
__global__ void __launch_bounds__(256, 2) k_bstencil_mma(float2* __restrict__ Y, const float2* __restrict__ X,
                                                         const float2* __restrict__ B, long vr,
                                                         const unsigned* __restrict__ Af, int Nx, int Nt, int ntiles,
                                                         Gate g) {
    extern __shared__ uint4 bst_op[];  // G sites x SITE_WORDS / 4
    constexpr int SITE_U4 = SITE_WORDS / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, t = lane & 3, p = gq & 1;
    const int nsite = Nx * Nt;
    const int G = ntiles >= 8 ? 1 : 8 / ntiles;
    const int sg = blockIdx.x * G;                 // first site of the group
    const int ng = min(G, nsite - sg);             // sites of the group
    // stage the group's operator
    const uint4* Ag = reinterpret_cast<const uint4*>(Af) + (long)sg * SITE_U4;
    const unsigned sbuf = (unsigned)__cvta_generic_to_shared(bst_op);
    for (int q = threadIdx.x; q < ng * SITE_U4; q += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbuf + 16u * q), "l"(Ag + q) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // this warp's task: site sg + warp / ntiles, tile warp % ntiles
    const int ls = warp / ntiles;
    const int r0 = (warp - ls * ntiles) * NB_TILE;
    const int s = sg + ls;
    const bool task = ls < ng && warp < G * ntiles;
    const bool run = task && __any_sync(0xffffffffu, gate_open(g, r0 + gq));
    float2 xv[5][3][2];
    if (run) {
        const float2* Xr = X + (long)(r0 + gq) * vr;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const float2* xn = Xr + (long)nbr_of(s, d, Nx, Nt) * NDOF;
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                xv[d][kt][0] = __ldg(xn + 8 * kt + t);
                xv[d][kt][1] = __ldg(xn + 8 * kt + t + 4);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (!run) return;
    float acc[3][4];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[m][i] = 0.f;
    const uint4* A4 = bst_op + ls * SITE_U4 + (gq >> 1) * 4 + t;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            const float2 x0 = xv[d][kt][0], x1 = xv[d][kt][1];
            const unsigned h0 = pack16<F16>(x0.x, x0.y), h1 = pack16<F16>(x1.x, x1.y);
            const float2 f0 = unpack16<F16>(h0), f1 = unpack16<F16>(h1);
            const unsigned l0 = pack16<F16>(x0.x - f0.x, x0.y - f0.y), l1 = pack16<F16>(x1.x - f1.x, x1.y - f1.y);
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                const uint4 w = A4[(d * 9 + mt * 3 + kt) * (TILE_WORDS / 4)];
                const unsigned a[4] = {embed(w.x, p), embed(w.y, p), embed(w.z, p), embed(w.w, p)};
                mma16816<F16>(acc[mt], a, h0, h1);
                mma16816<F16>(acc[mt], a, l0, l1);
            }
        }
    }
    // lane (gq, t) holds component p of outputs a = gq / 2 and a + 4 for right-hand
    // sides r0 + 2t, r0 + 2t + 1; lane ^ 4 holds the other component
#pragma unroll
    for (int mt = 0; mt < 3; ++mt) {
        const float s0 = p ? acc[mt][0] : acc[mt][2], s1 = p ? acc[mt][1] : acc[mt][3];
        const float o0 = __shfl_xor_sync(0xffffffffu, s0, 4), o1 = __shfl_xor_sync(0xffffffffu, s1, 4);
        const int row = 8 * mt + (gq >> 1) + (p ? 4 : 0);
        float2 v[2];
        v[0] = p ? make_float2(o0, acc[mt][2]) : make_float2(acc[mt][0], o0);
        v[1] = p ? make_float2(o1, acc[mt][3]) : make_float2(acc[mt][1], o1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = r0 + 2 * t + q;
            if (!gate_open(g, r)) continue;
            const long off = (long)r * vr + (long)s * NDOF + row;
            float2 o = v[q];
            if (RES) {
                const float2 bb = __ldg(B + off);
                o = make_float2(bb.x - o.x, bb.y - o.y);
            }
            Y[off] = o;
        }
    }
}

}  // namespace

// ------------------------------------------------------------- launchers ----

template <typename T>
void launch_bgram(double2* out, long os, const C2<T>* V, long ldv, long vr, int nd, const int* ndd, long nds,
                  const C2<T>* w, long wr, long n, int nb, BRed red, Gate g, cudaStream_t s) {
    if (nd <= 0 && !ndd) return;
    const int ch = chunks_for(n, red);
    k_bgram<T><<<dim3(ch, nb), BT, 0, s>>>(out, os, V, ldv, vr, nd, ndd, nds, w, wr, n,
                                           reinterpret_cast<C2<T>*>(red.partial), red.max_chunks, red.ticket, g);
    count_launch();
}

template <typename T>
void launch_baxpy(C2<T>* w, long wr, const C2<T>* V, long ldv, long vr, int nd, const int* ndd, long nds,
                  const double2* coef, long cs, double sign, bool zero_first, long n, int nb, double* norm2,
                  long n2s, BRed red, Gate g, cudaStream_t s) {
    const int ch = chunks_for(n, red);
    k_baxpy<T><<<dim3(ch, nb), BT, 0, s>>>(w, wr, V, ldv, vr, nd, ndd, nds, coef, cs, sign, zero_first ? 1 : 0, n,
                                           norm2, n2s, reinterpret_cast<C2<T>*>(red.partial), red.max_chunks,
                                           red.ticket, g);
    count_launch();
}

template <typename T>
void launch_bnorm2(double* out, long os, const C2<T>* v, long vr, long n, int nb, BRed red, Gate g, cudaStream_t s) {
    const int ch = chunks_for(n, red);
    k_bnorm2<T><<<dim3(ch, nb), BT, 0, s>>>(out, os, v, vr, n, reinterpret_cast<C2<T>*>(red.partial), red.max_chunks,
                                            red.ticket, g);
    count_launch();
}

template <typename T>
void launch_bscale(C2<T>* y, long yr, const C2<T>* x, long xr, const double* f, long fs, long n, int nb, Gate g,
                   cudaStream_t s) {
    k_bscale<T><<<dim3(ew_chunks(n), nb), 256, 0, s>>>(y, yr, x, xr, f, fs, n, g);
    count_launch();
}

template <typename Ta, typename Tb>
void launch_bconvert(C2<Tb>* y, long yr, const C2<Ta>* x, long xr, long n, int nb, cudaStream_t s) {
    k_bconvert<Ta, Tb><<<dim3(ew_chunks(n), nb), 256, 0, s>>>(y, yr, x, xr, n);
    count_launch();
}

void launch_pack_frag(unsigned* out, const double2* A, long nsite, bool fp16, cudaStream_t s) {
    const long total = nsite * SITE_WORDS;
    const unsigned grid = (unsigned)std::min<long>((total + 255) / 256, (long)sm_count() * 16);
    if (fp16) k_pack_frag<true><<<grid, 256, 0, s>>>(out, A, nsite);
    else k_pack_frag<false><<<grid, 256, 0, s>>>(out, A, nsite);
    count_launch();
}

void launch_bstencil_mma(float2* Y, const float2* X, const float2* B, long vr, const unsigned* Af, int Nx, int Nt,
                         int nb, bool fp16, Gate g, cudaStream_t s) {
    const int ntiles = nb / NB_TILE;
    const int G = ntiles >= 8 ? 1 : 8 / ntiles;  // sites per CTA
    const long nsite = (long)Nx * Nt;
    const unsigned grid = (unsigned)((nsite + G - 1) / G);
    const size_t smem = (size_t)G * SITE_WORDS * sizeof(unsigned);
    static bool attr_set[64] = {};  // larger than the default 48 KB when G > 4
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
        const int mx = 8 * SITE_WORDS * (int)sizeof(unsigned);
        cudaFuncSetAttribute(k_bstencil_mma<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_bstencil_mma<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_bstencil_mma<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_bstencil_mma<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr_set[dev] = true;
    }
    if (fp16) {
        if (B) k_bstencil_mma<true, true><<<grid, 256, smem, s>>>(Y, X, B, vr, Af, Nx, Nt, ntiles, g);
        else k_bstencil_mma<true, false><<<grid, 256, smem, s>>>(Y, X, B, vr, Af, Nx, Nt, ntiles, g);
    } else {
        if (B) k_bstencil_mma<false, true><<<grid, 256, smem, s>>>(Y, X, B, vr, Af, Nx, Nt, ntiles, g);
        else k_bstencil_mma<false, false><<<grid, 256, smem, s>>>(Y, X, B, vr, Af, Nx, Nt, ntiles, g);
    }
    count_launch();
}

#define INST(T)                                                                                                     \
    template void launch_bgram<T>(double2*, long, const C2<T>*, long, long, int, const int*, long, const C2<T>*,    \
                                  long, long, int, BRed, Gate, cudaStream_t);                                      \
    template void launch_baxpy<T>(C2<T>*, long, const C2<T>*, long, long, int, const int*, long, const double2*,    \
                                  long, double, bool, long, int, double*, long, BRed, Gate, cudaStream_t);         \
    template void launch_bnorm2<T>(double*, long, const C2<T>*, long, long, int, BRed, Gate, cudaStream_t);         \
    template void launch_bscale<T>(C2<T>*, long, const C2<T>*, long, const double*, long, long, int, Gate,          \
                                   cudaStream_t);
INST(double)
INST(float)
#undef INST
template void launch_bconvert<double, float>(C2<float>*, long, const C2<double>*, long, long, int, cudaStream_t);
template void launch_bconvert<float, double>(C2<double>*, long, const C2<float>*, long, long, int, cudaStream_t);

}  // namespace mg
