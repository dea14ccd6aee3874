// The Arnoldi steps of the batched coarse GMRES-Proj (Section 2) for a block of
// right-hand sides.  Work is split over (site chunk) x (tile of eight
// right-hand sides); a step has three phases:
//   S1  w = A v_j on the chunk's sites (tensor-core block products, as in the
//       block stencil of batch.cu) and the chunk's partial sums of V^+ w; the
//       last chunk of a tile to finish adds the partials in chunk order (h1);
//   S2  w -= V h1, and partial sums of V^+ w and ||w||^2 from the same pass
//       over the basis; the last chunk of a tile adds them (h2, ||w||^2), forms
//       h_{j+1,j} = sqrt(||w||^2 - ||h2||^2) (the basis is orthonormal, as in the
//       single-right-hand-side cluster kernel) and pushes column j into the FP64
//       least squares of each right-hand side;
//   S3  v_{j+1} = (w - V h2) / h_{j+1,j}.
// Two forms run them.  The cycle kernel (k_cb_cycle) keeps every CTA of the
// block resident (cooperative launch) and runs all steps of a GMRES cycle: the
// CTAs of a tile meet at a bounded tile barrier after each phase, and each CTA
// adds the chunk partials of its right-hand sides itself.  The step kernels
// (one launch per phase, the last chunk of a tile to finish does the adds) serve
// coarse grids whose chunking does not fit the resident grid.
// The step gate of a right-hand side is double-buffered by step parity: the
// push of step j writes the gate that step j + 1 reads, while every CTA of step
// j reads the buffer of step j.  The basis rows are V[i][r][n] (FP32).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "batch.cuh"
#include "coarse_block.cuh"
#include "ks_dev.cuh"

namespace mg {

namespace {

constexpr int NDOF = 24;
constexpr int TILE_WORDS = 64;
constexpr int SITE_WORDS = 5 * 9 * TILE_WORDS;
constexpr int MAXI = MSMAX + 1;  // basis vectors of a cycle
#ifndef CB_APPLY_MT
#define CB_APPLY_MT 3  // output tiles per apply task of the cycle kernel (1 or 3)
#endif
#ifndef CB_COOP_MINB
#define CB_COOP_MINB 1  // resident cycle-kernel CTAs per SM the register budget is sized for
#endif

template <bool F16>
__device__ __forceinline__ unsigned pk(float re, float im) {
    if constexpr (F16) {
        const __half2 h = __floats2half2_rn(re, im);
        return *reinterpret_cast<const unsigned*>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        return *reinterpret_cast<const unsigned*>(&h);
    }
}
template <bool F16>
__device__ __forceinline__ float2 upk(unsigned u) {
    if constexpr (F16) return __half22float2(*reinterpret_cast<const __half2*>(&u));
    else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
template <bool F16>
__device__ __forceinline__ void mma(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    if constexpr (F16)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    else
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
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

__device__ __forceinline__ float2 warp_sum2(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

__device__ __forceinline__ float2* part_slot(float2* part, int r, int i, int c) {
    return part + ((long)r * CB_PB + i) * CB_MAXCH + c;
}

// true in every thread of the CTA that is the last of the nchunks CTAs of its
// tile to arrive (after each has written its partial sums)
__device__ __forceinline__ bool last_chunk(unsigned* ticket, int nchunks) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)nchunks - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Reduction scratch of one warp: v[i][lane] holds lane's value g0 + i of a
// group of 16 values.
struct WarpRed {
    float2 v[16][32];
};

// Sum over the lanes of each value i < nv held per lane in acc, 16 values at a
// time: the lanes store them, then lane i adds row i in lane order (a fixed
// order: the same result in every CTA).  Returns the total of value `lane`
// (lanes >= nv: zero).
template <int JB>
__device__ __forceinline__ float2 lane_sums(const float2 (&acc)[JB], int nv, WarpRed& red) {
    const int lane = threadIdx.x & 31;
    float2 t = make_float2(0.f, 0.f);
#pragma unroll
    for (int g0 = 0; g0 < JB; g0 += 16) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (g0 + i < JB && g0 + i < nv) red.v[i][lane] = acc[g0 + i < JB ? g0 + i : 0];
        __syncwarp();
        if (lane >= g0 && lane < g0 + 16 && lane < nv)
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                const float2 b = red.v[lane - g0][q];
                t.x += b.x;
                t.y += b.y;
            }
        __syncwarp();
    }
    return t;
}

// dynamic shared memory of the coarse step kernels and the cycle kernel
struct CBSmem {
    float2 ws[NB_TILE][CB_MAXSPC * NDOF];  // w of the chunk's sites, per right-hand side
    float2 hs[NB_TILE][MAXI];              // reduced products of the current pass
    float hn[NB_TILE];                     // h_{j+1,j} per right-hand side
    WarpRed red[NB_TILE + 1];
};

// dynamic shared memory of the cycle kernel (CB_WPR warps per right-hand side);
// it is followed by w of the chunk's sites, NB_TILE rows of spc * NDOF entries
// (sized at launch, so larger coarse grids can take larger chunks)
struct CBCycleSmem {
    float2 hs[NB_TILE * CB_WPR][MAXI];
    float2 h1[NB_TILE][MAXI];      // chunk 0: first-pass products kept for the push
    float hn[NB_TILE];
    // chunk 0: the least squares of each right-hand side during the cycle (FP64):
    // rotations, the rotated right-hand side, the tolerance, and a column
    double rc[NB_TILE][MSMAX];
    double2 rs[NB_TILE][MSMAX];
    double2 g[NB_TILE][MSMAX + 1];
    double2 col[NB_TILE][MAXI + 1];
    double tol[NB_TILE];
    WarpRed red[NB_TILE * CB_WPR];
    uint4 abuf[NB_TILE * CB_WPR][SITE_WORDS / 4];  // each warp's staged operator tiles of one site
};

// Column jh of right-hand side r's least squares (the cycle kernel's push): the
// column h1 + h2 with subdiagonal hn, rotated by the cycle's earlier rotations
// (kept in shared memory, so no step waits on a dependent global load), a new
// rotation, the rotated right-hand side, the residual estimate and the gates.
// The state in global memory receives what the cycle's finish reads (H, R, g,
// rotations, j, res, conv) without being read back.
__device__ __forceinline__ void push_cycle(const CBArgs& a, CBCycleSmem& S, int l, int r, int jh, const float2* h2) {
    KState* ks = a.ks + r;
    double2* col = S.col[l];
    for (int i = 0; i <= jh; ++i) col[i] = make_double2((double)S.h1[l][i].x + (double)h2[i].x,
                                                        (double)S.h1[l][i].y + (double)h2[i].y);
    const double hn = (double)S.hn[l];
    col[jh + 1] = make_double2(hn, 0.0);
    double2* Hc = ks->H + KLD * jh;
    double2* Rc = ks->R + KLD * jh;
    for (int i = 0; i <= jh + 1; ++i) Hc[i] = col[i];
    for (int i = jh + 2; i < KLD; ++i) {
        Hc[i] = make_double2(0.0, 0.0);
        Rc[i] = make_double2(0.0, 0.0);
    }
    double2 p = col[0];
    for (int t = 0; t < jh; ++t) {
        double2 q = col[t + 1];
        ksd::rot_apply(S.rc[l][t], S.rs[l][t], p, q);
        Rc[t] = p;
        p = q;
    }
    double cc;
    double2 ss, rr;
    ksd::givens(p, col[jh + 1], cc, ss, rr);
    Rc[jh] = rr;
    Rc[jh + 1] = make_double2(0.0, 0.0);
    S.rc[l][jh] = cc;
    S.rs[l][jh] = ss;
    ks->rc[jh] = cc;
    ks->rs[jh] = ss;
    ks->ra[jh] = (short)jh;
    ks->rb[jh] = (short)(jh + 1);
    ksd::rot_apply(cc, ss, S.g[l][jh], S.g[l][jh + 1]);
    ks->g[jh] = S.g[l][jh];
    ks->g[jh + 1] = S.g[l][jh + 1];
    const double res = ksd::cabsd(S.g[l][jh + 1]);
    const int conv = res <= S.tol[l] ? 1 : 0, brk = hn == 0.0 ? 1 : 0;
    const int next = (conv || brk || jh + 1 >= KMAX) ? -1 : jh + 1;
    ks->nrot = jh + 1;
    ks->res = res;
    ks->j = jh + 1;
    ks->conv = conv;
    ks->breakdown = brk;
    ks->step_gate = next;
    ks->scale_gate = hn > 0.0 ? jh + 1 : -1;
    ks->scale = hn > 0.0 ? 1.0 / hn : 0.0;
    a.gbuf[((jh + 1) & 1) * a.nbp + r] = next;
}

// slots 0..jh (and, with norm, slot CB_PB - 1) of right-hand side r summed over
// the chunks: lanes over the chunks in a fixed order, then lane_sums.  Lane i
// returns slot i's total (i <= jh); with norm, *nrm is the norm's total in every
// lane.
template <int JB>
__device__ __forceinline__ float2 chunk_totals(const float2* part, int nchunks, int r, int jh, bool norm, float* nrm,
                                               WarpRed& red) {
    const float2* p = part + (long)r * CB_PB * CB_MAXCH;
    const int lane = threadIdx.x & 31;
    float2 v[JB];
    float nv = 0.f;
#pragma unroll
    for (int i = 0; i < JB; ++i) v[i] = make_float2(0.f, 0.f);
    for (int cc = lane; cc < nchunks; cc += 32) {
#pragma unroll
        for (int i = 0; i < JB; ++i)
            if (i <= jh) {
                const float2 b = __ldcg(p + (long)i * CB_MAXCH + cc);
                v[i].x += b.x;
                v[i].y += b.y;
            }
        if (norm) nv += __ldcg(p + (long)(CB_PB - 1) * CB_MAXCH + cc).x;
    }
    if (norm) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
        *nrm = nv;
    }
    return lane_sums<JB>(v, jh + 1, red);
}


// ---------------------------------------------------------------- phases ----

// w = A v_jh on the chunk's sites for the tile's eight right-hand sides (into
// ws and, for right-hand sides whose bit is set in `wmask`, into V[jh+1]).  One
// warp task per (site, MT consecutive 8-row tiles of the output): MT = 3 covers
// a site with one pass over its neighbour values; the next direction's operator
// tiles and neighbour values load while this one multiplies.  nwarps warps take
// part.
template <bool F16, int MT>
__device__ __forceinline__ void phase_apply(const CBArgs& a, int jh, int r0, int s0, int ns, unsigned wmask,
                                            float2 (*ws)[CB_MAXSPC * NDOF], int nwarps) {
    constexpr int NT = 3 / MT;  // tasks per site
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, t = lane & 3, p = gq & 1;
    const float2* X = a.V + (long)jh * a.row;
    float2* Wt = a.V + (long)(jh + 1) * a.row;
    for (int task = warp; task < ns * NT; task += nwarps) {
        const int ls = task / NT, mt0 = (task - NT * ls) * MT;
        const int s = s0 + ls;
        float acc[MT][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[m][i] = 0.f;
        const uint4* A4 = reinterpret_cast<const uint4*>(a.Af) + (long)s * (SITE_WORDS / 4) + (gq >> 1) * 4 + t +
                          mt0 * 3 * (TILE_WORDS / 4);
        const float2* Xr = X + (long)(r0 + gq) * a.n;
        float2 xv[3][2];
        uint4 aw[MT][3];
        auto load = [&](int d) {
            const float2* xn = Xr + (long)nbr_of(s, d, a.Nx, a.Nt) * NDOF;
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                xv[kt][0] = __ldcg(xn + 8 * kt + t);
                xv[kt][1] = __ldcg(xn + 8 * kt + t + 4);
#pragma unroll
                for (int m = 0; m < MT; ++m) aw[m][kt] = __ldg(A4 + (d * 9 + m * 3 + kt) * (TILE_WORDS / 4));
            }
        };
        load(0);
#pragma unroll 1
        for (int d = 0; d < 5; ++d) {
            float2 xc[3][2];
            uint4 ac[MT][3];
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                xc[kt][0] = xv[kt][0];
                xc[kt][1] = xv[kt][1];
#pragma unroll
                for (int m = 0; m < MT; ++m) ac[m][kt] = aw[m][kt];
            }
            if (d < 4) load(d + 1);
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                const float2 x0 = xc[kt][0], x1 = xc[kt][1];
                const unsigned h0 = pk<F16>(x0.x, x0.y), h1 = pk<F16>(x1.x, x1.y);
                const float2 f0 = upk<F16>(h0), f1 = upk<F16>(h1);
                const unsigned l0 = pk<F16>(x0.x - f0.x, x0.y - f0.y), l1 = pk<F16>(x1.x - f1.x, x1.y - f1.y);
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    const uint4 w = ac[m][kt];
                    const unsigned av[4] = {embed(w.x, p), embed(w.y, p), embed(w.z, p), embed(w.w, p)};
                    mma<F16>(acc[m], av, h0, h1);
                    mma<F16>(acc[m], av, l0, l1);
                }
            }
        }
        // lane (gq, t) holds component p of outputs gq / 2 and gq / 2 + 4 of
        // right-hand sides 2t, 2t + 1; lane ^ 4 holds the other component
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const float s0v = p ? acc[m][0] : acc[m][2], s1v = p ? acc[m][1] : acc[m][3];
            const float o0 = __shfl_xor_sync(0xffffffffu, s0v, 4), o1 = __shfl_xor_sync(0xffffffffu, s1v, 4);
            const int row = 8 * (mt0 + m) + (gq >> 1) + (p ? 4 : 0);
            const float2 v0 = p ? make_float2(o0, acc[m][2]) : make_float2(acc[m][0], o0);
            const float2 v1 = p ? make_float2(o1, acc[m][3]) : make_float2(acc[m][1], o1);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int rl = 2 * t + q;
                const float2 v = q ? v1 : v0;
                ws[rl][ls * NDOF + row] = v;
                if ((wmask >> rl) & 1u) Wt[(long)(r0 + rl) * a.n + (long)s * NDOF + row] = v;
            }
        }
    }
}

// The cycle kernel's apply: one warp task per site (all three output tiles).
// The site's operator tiles (5 x 9 x 256 bytes) go to the warp's shared buffer
// by 16-byte asynchronous copies, and the neighbour values of all five
// directions to registers, all issued at once: one memory latency per site.
template <bool F16>
__device__ __forceinline__ void phase_apply_staged(const CBArgs& a, int jh, int r0, int s0, int ns, unsigned wmask,
                                                   float2* ws, int wst, uint4* abuf, int nwarps) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, t = lane & 3, p = gq & 1;
    const float2* X = a.V + (long)jh * a.row;
    float2* Wt = a.V + (long)(jh + 1) * a.row;
    constexpr int SITE_U4 = SITE_WORDS / 4;  // 720 sixteen-byte pieces
    const unsigned sbuf = (unsigned)__cvta_generic_to_shared(abuf);
    for (int ls = warp; ls < ns; ls += nwarps) {
        const int s = s0 + ls;
        const uint4* Ag = reinterpret_cast<const uint4*>(a.Af) + (long)s * SITE_U4;
        __syncwarp();  // the previous site's reads of the buffer are done
        for (int q = lane; q < SITE_U4; q += 32)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbuf + 16u * q), "l"(Ag + q) : "memory");
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const float2* Xr = X + (long)(r0 + gq) * a.n;
        float2 xv[5][3][2];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const float2* xn = Xr + (long)nbr_of(s, d, a.Nx, a.Nt) * NDOF;
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                xv[d][kt][0] = __ldcg(xn + 8 * kt + t);
                xv[d][kt][1] = __ldcg(xn + 8 * kt + t + 4);
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncwarp();
        float acc[3][4];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[m][i] = 0.f;
        const uint4* A4 = abuf + (gq >> 1) * 4 + t;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
#pragma unroll
            for (int kt = 0; kt < 3; ++kt) {
                const float2 x0 = xv[d][kt][0], x1 = xv[d][kt][1];
                const unsigned h0 = pk<F16>(x0.x, x0.y), h1 = pk<F16>(x1.x, x1.y);
                const float2 f0 = upk<F16>(h0), f1 = upk<F16>(h1);
                const unsigned l0 = pk<F16>(x0.x - f0.x, x0.y - f0.y), l1 = pk<F16>(x1.x - f1.x, x1.y - f1.y);
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const uint4 w = A4[(d * 9 + m * 3 + kt) * (TILE_WORDS / 4)];
                    const unsigned av[4] = {embed(w.x, p), embed(w.y, p), embed(w.z, p), embed(w.w, p)};
                    mma<F16>(acc[m], av, h0, h1);
                    mma<F16>(acc[m], av, l0, l1);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float s0v = p ? acc[m][0] : acc[m][2], s1v = p ? acc[m][1] : acc[m][3];
            const float o0 = __shfl_xor_sync(0xffffffffu, s0v, 4), o1 = __shfl_xor_sync(0xffffffffu, s1v, 4);
            const int row = 8 * m + (gq >> 1) + (p ? 4 : 0);
            const float2 v0 = p ? make_float2(o0, acc[m][2]) : make_float2(acc[m][0], o0);
            const float2 v1 = p ? make_float2(o1, acc[m][3]) : make_float2(acc[m][1], o1);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int rl = 2 * t + q;
                const float2 v = q ? v1 : v0;
                ws[rl * wst + ls * NDOF + row] = v;
                if ((wmask >> rl) & 1u) Wt[(long)(r0 + rl) * a.n + (long)s * NDOF + row] = v;
            }
        }
    }
}

// the bits of the tile's right-hand sides whose gate opens step jh
__device__ __forceinline__ unsigned gate_mask(const int* gate, int r0, int jh) {
    unsigned m = 0u;
#pragma unroll
    for (int q = 0; q < NB_TILE; ++q) m |= (__ldcg(gate + r0 + q) == jh ? 1u : 0u) << q;
    return m;
}

// partial sums over the chunk of V^+ w (w in ws) for right-hand side r, one
// warp; JB >= jh + 1 bounds the rows at compile time
// Elements e0, e0 + es, ... of the chunk; slot: this warp's partial-sum slot.
// For JB <= 16 two elements per iteration, so twice the loads are in flight.
template <int JB>
__device__ __forceinline__ void phase_gram1(const CBArgs& a, int jh, int r, int slot, int s0, int ne, int e0, int es,
                                            const float2* wsr, WarpRed& red) {
    constexpr int U = JB <= 16 ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const float2* Vr = a.V + (long)r * a.n + (long)s0 * NDOF;
    float2 acc[JB];
#pragma unroll
    for (int i = 0; i < JB; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int e = e0; e < ne; e += U * es) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int eu = e + u * es;
            if (eu < ne) {
                const float2 we = wsr[eu];
#pragma unroll
                for (int i = 0; i < JB; ++i)
                    if (i <= jh) acc[i] = cfmac(__ldcg(Vr + (long)i * a.row + eu), we, acc[i]);
            }
        }
    }
    const float2 t = lane_sums<JB>(acc, jh + 1, red);
    if (lane <= jh) *part_slot(a.p1, r, lane, slot) = t;
}

// w -= V h1 (h1 in hs) on the chunk, and partial sums of V^+ w and ||w||^2, one
// warp.  The chunk's basis rows are written only by this CTA; NC: they were
// written by an earlier launch, so the read-only path may cache them.
template <bool NC, int JB>
__device__ __forceinline__ void phase_update_gram(const CBArgs& a, int jh, int r, int slot, int s0, int ne, int e0,
                                                  int es, const float2* hs, WarpRed& red) {
    const int lane = threadIdx.x & 31;
    const float2* Vr = a.V + (long)r * a.n + (long)s0 * NDOF;
    float2* w = a.V + (long)(jh + 1) * a.row + (long)r * a.n + (long)s0 * NDOF;
    float2 acc[JB];
#pragma unroll
    for (int i = 0; i < JB; ++i) acc[i] = make_float2(0.f, 0.f);
    float nn = 0.f;
    for (int e = e0; e < ne; e += es) {
        float2 wv = __ldcg(w + e);
        // rows 0..jh are not written in this phase: the second pass finds them in L1
#pragma unroll
        for (int i = 0; i < JB; ++i)
            if (i <= jh) {
                const float2 vi = NC ? __ldg(Vr + (long)i * a.row + e) : Vr[(long)i * a.row + e];
                const float2 h = hs[i];
                wv.x -= vi.x * h.x - vi.y * h.y;
                wv.y -= vi.x * h.y + vi.y * h.x;
            }
#pragma unroll
        for (int i = 0; i < JB; ++i)
            if (i <= jh) acc[i] = cfmac(NC ? __ldg(Vr + (long)i * a.row + e) : Vr[(long)i * a.row + e], wv, acc[i]);
        nn += wv.x * wv.x + wv.y * wv.y;
        w[e] = wv;
    }
    const float2 t = lane_sums<JB>(acc, jh + 1, red);
    if (lane <= jh) *part_slot(a.p2, r, lane, slot) = t;
    const float2 nv = warp_sum2(make_float2(nn, 0.f));
    if (lane == 0) *part_slot(a.p2, r, CB_PB - 1, slot) = nv;
}

// v_{jh+1} = (w - V h2) * inv on the chunk (h2 in hs), one warp
template <int JB>
__device__ __forceinline__ void phase_update(const CBArgs& a, int jh, int r, int s0, int ne, int e0, int es,
                                             const float2* hs, float inv) {
    constexpr int U = JB <= 16 ? 2 : 1;
    const float2* Vr = a.V + (long)r * a.n + (long)s0 * NDOF;
    float2* w = a.V + (long)(jh + 1) * a.row + (long)r * a.n + (long)s0 * NDOF;
    for (int e = e0; e < ne; e += U * es) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int eu = e + u * es;
            if (eu < ne) {
                float2 wv = __ldcg(w + eu);
#pragma unroll
                for (int i = 0; i < JB; ++i)
                    if (i <= jh) {
                        const float2 vi = __ldcg(Vr + (long)i * a.row + eu);
                        const float2 h = hs[i];
                        wv.x -= vi.x * h.x - vi.y * h.y;
                        wv.y -= vi.x * h.y + vi.y * h.x;
                    }
                w[eu] = make_float2(wv.x * inv, wv.y * inv);
            }
        }
    }
}

// from lane i's total t of h2_i (lanes <= jh) and ||w||^2:
// h_{j+1,j} = ||w - V h2|| = sqrt(||w||^2 - ||h2||^2) (the basis is orthonormal),
// the same in every lane
__device__ __forceinline__ float subdiag(float2 t, int jh, float nrm) {
    const int lane = threadIdx.x & 31;
    float h2n = lane <= jh ? t.x * t.x + t.y * t.y : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h2n += __shfl_xor_sync(0xffffffffu, h2n, o);
    return sqrtf(fmaxf(nrm - h2n, 0.f));
}

// dispatch on the rows of step jh: compile-time bounds 8, 16 and MAXI
#define CB_DISPATCH(jh, CALL) \
    do {                      \
        if ((jh) < 8) {       \
            constexpr int JB = 8; \
            CALL;             \
        } else if ((jh) < 16) { \
            constexpr int JB = 16; \
            CALL;             \
        } else {              \
            constexpr int JB = MAXI; \
            CALL;             \
        }                     \
    } while (0)

// column jh into the FP64 least squares of right-hand side r and its next gate
// (hA and hB already in the state)
__device__ __forceinline__ void push_column(const CBArgs& a, int jh, int r, float hn) {
    KState* ks = a.ks + r;
    ks->hn2 = (double)hn * (double)hn;
    ksd::ks_push_dev(ks, jh);
    a.gbuf[((jh + 1) & 1) * a.nbp + r] = ks->step_gate;
}

// ---------------------------------------------------------- step kernels ----

template <bool F16>
__global__ void __launch_bounds__(CB_THREADS, 2) k_cb_apply_gram(CBArgs a, int jh) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    CBSmem& S = *reinterpret_cast<CBSmem*>(cb_smem);
    auto& ws = S.ws;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.y * NB_TILE, c = blockIdx.x;
    const int nsite = a.Nx * a.Nt;
    const int s0 = c * a.spc;
    const int ns = min(a.spc, nsite - s0);
    const int* gate = a.gbuf + (jh & 1) * a.nbp;
    if (!__syncthreads_or(threadIdx.x < NB_TILE && __ldcg(gate + r0 + threadIdx.x) == jh)) return;
    phase_apply<F16, 1>(a, jh, r0, s0, ns, gate_mask(gate, r0, jh), ws, CB_THREADS / 32);
    __syncthreads();
    const int r = r0 + warp;
    const bool on = __ldcg(gate + r) == jh;
    if (on) CB_DISPATCH(jh, (phase_gram1<JB>(a, jh, r, c, s0, ns * NDOF, lane, 32, ws[warp], S.red[warp])));
    // the last chunk of the tile adds the partials: h1 of every right-hand side
    if (!last_chunk(a.ticket + blockIdx.y, a.nchunks)) return;
    if (on) {
        float2 t;
        CB_DISPATCH(jh, (t = chunk_totals<JB>(a.p1, a.nchunks, r, jh, false, nullptr, S.red[warp])));
        if (lane <= jh) {
            a.h1[(long)r * CB_PB + lane] = t;
            a.ks[r].hA[lane] = make_double2(t.x, t.y);
        }
    }
    if (threadIdx.x == 0) a.ticket[blockIdx.y] = 0u;
}

__global__ void __launch_bounds__(CB_THREADS, 2) k_cb_update_gram(CBArgs a, int jh) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    CBSmem& S = *reinterpret_cast<CBSmem*>(cb_smem);
    auto& hs = S.hs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.y * NB_TILE, c = blockIdx.x;
    const int* gate = a.gbuf + (jh & 1) * a.nbp;
    if (!__syncthreads_or(threadIdx.x < NB_TILE && __ldcg(gate + r0 + threadIdx.x) == jh)) return;
    const int r = r0 + warp;
    const bool on = __ldcg(gate + r) == jh;
    const int nsite = a.Nx * a.Nt;
    const int s0 = c * a.spc;
    const int ns = min(a.spc, nsite - s0);
    if (on) {
        if (lane <= jh) hs[warp][lane] = __ldcg(a.h1 + (long)r * CB_PB + lane);
        __syncwarp();
        CB_DISPATCH(jh, (phase_update_gram<true, JB>(a, jh, r, c, s0, ns * NDOF, lane, 32, hs[warp], S.red[warp])));
    }
    // the last chunk of the tile: h2, ||w||^2, h_{j+1,j}, and the least-squares push
    if (!last_chunk(a.ticket + a.nbp / NB_TILE + blockIdx.y, a.nchunks)) return;
    if (on) {
        float2 t;
        float nrm = 0.f;
        CB_DISPATCH(jh, (t = chunk_totals<JB>(a.p2, a.nchunks, r, jh, true, &nrm, S.red[warp])));
        const float hn = subdiag(t, jh, nrm);
        if (lane <= jh) {
            a.h2[(long)r * CB_PB + lane] = t;
            a.ks[r].hB[lane] = make_double2(t.x, t.y);
        }
        __syncwarp();
        if (lane == 0) {
            a.h2[(long)r * CB_PB + CB_PB - 1] = make_float2(hn, hn > 0.f ? 1.f / hn : 0.f);
            push_column(a, jh, r, hn);
        }
    }
    if (threadIdx.x == 0) a.ticket[a.nbp / NB_TILE + blockIdx.y] = 0u;
}

// v_{j+1} = (w - V h2) / h_{j+1,j}
__global__ void __launch_bounds__(CB_THREADS, 2) k_cb_update_push(CBArgs a, int jh) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    CBSmem& S = *reinterpret_cast<CBSmem*>(cb_smem);
    auto& hs = S.hs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y * NB_TILE + warp, c = blockIdx.x;
    if (__ldcg(a.gbuf + (jh & 1) * a.nbp + r) != jh) return;
    const int nsite = a.Nx * a.Nt;
    const int s0 = c * a.spc;
    const int ns = min(a.spc, nsite - s0);
    if (lane <= jh) hs[warp][lane] = __ldcg(a.h2 + (long)r * CB_PB + lane);
    const float inv = __ldcg(a.h2 + (long)r * CB_PB + CB_PB - 1).y;
    __syncwarp();
    CB_DISPATCH(jh, (phase_update<JB>(a, jh, r, s0, ns * NDOF, lane, 32, hs[warp], inv)));
}

// ---------------------------------------------------------- cycle kernel ----

// Barrier of the nchunks CTAs of one tile, bounded: the generation is read
// before arriving, the last arrival resets the count and advances the
// generation, the others wait (at most `spin` polls) for it to change.  A wait
// that gives up sets *err; the CTA then goes on, so every barrier still ends.
__device__ __forceinline__ void tile_sync(unsigned* bar, unsigned n, long spin, int* err) {
    __syncthreads();  // the CTA's writes of the phase precede thread 0's release below
    if (threadIdx.x == 0) {
        unsigned* gen = bar + 1;
        unsigned g, old;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(g) : "l"(gen) : "memory");
        // arrival: release this CTA's writes, acquire the earlier arrivals' ones
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;\n" : "=r"(old) : "l"(bar) : "memory");
        if (old == n - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;\n" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(gen) : "memory");
        } else {
            long it = 0;
            unsigned cur;
            while (true) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(cur) : "l"(gen) : "memory");
                if (cur != g) break;
                if (++it > spin) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();  // thread 0's acquire orders the other arrivals' writes before every thread's reads
}

#ifdef CB_PHASE_CLOCKS
// phase timing of CTA (0, 0) (a build with -DCB_PHASE_CLOCKS): per step the time
// to the end of each phase's own work and of each barrier, printed for the first
// launches
__device__ unsigned cb_clock_launches = 0;
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define CB_STAMP(k)                                        \
    do {                                                   \
        if (clk && threadIdx.x == 0) {                     \
            const unsigned long long now = gtime();        \
            acc_t[k] += now - t_prev;                      \
            t_prev = now;                                  \
        }                                                  \
    } while (0)
#else
#define CB_STAMP(k) \
    do {            \
    } while (0)
#endif

// All ms steps of one GMRES cycle for every right-hand side of the block; the
// grid (chunks x tiles) is resident at once (cooperative launch).  Warps 0..7
// own the tile's right-hand sides; warp 8 pushes the least-squares columns of
// the tile (in the CTA of chunk 0) while warps 0..7 form v_{j+1}.
template <bool F16>
__global__ void __launch_bounds__(CB_COOP_THREADS, CB_COOP_MINB) k_cb_cycle(CBArgs a, int ms, long spin, int* err) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    CBCycleSmem& S = *reinterpret_cast<CBCycleSmem*>(cb_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.y, r0 = tile * NB_TILE, c = blockIdx.x;
    const int nsite = a.Nx * a.Nt;
    const int s0 = c * a.spc;
    const int ns = min(a.spc, nsite - s0);
    const int ne = ns * NDOF;
    unsigned* bar = a.bar + 2 * tile;
    // warps 0 .. 8 CB_WPR - 1: right-hand side r0 + (warp % 8), element part warp / 8
    // (its own partial-sum slot); warp 8 CB_WPR: the pushes of chunk 0
    constexpr int NRW = NB_TILE * CB_WPR;
    const bool rw = warp < NRW;
    const int rl = warp % NB_TILE, part = warp / NB_TILE;
    const int r = r0 + rl;
    const int slot = c * CB_WPR + part, nslot = a.nchunks * CB_WPR;
    const int e0 = part * 32 + lane, es = 32 * CB_WPR;
    const int wst = a.spc * NDOF;
    float2* wsb = reinterpret_cast<float2*>(cb_smem + sizeof(CBCycleSmem));
#ifdef CB_PHASE_CLOCKS
    __shared__ unsigned clk_s;
    if (threadIdx.x == 0) clk_s = (c == 0 && tile == 0) ? atomicAdd(&cb_clock_launches, 1u) < 3 : 0;
    __syncthreads();
    const bool clk = clk_s != 0;
    unsigned long long acc_t[7] = {0, 0, 0, 0, 0, 0, 0}, t_prev = gtime();
    int steps = 0;
#endif
    if (a.probe && threadIdx.x == 0) {  // test probe: a wait that nothing ends gives up
        const volatile unsigned* never = a.bar + 2 * (NB_MAX / NB_TILE);
        long it = 0;
        while (*never == 0u) {
            if (++it > spin) {
                atomicExch(err, 1);
                break;
            }
            __nanosleep(32);
        }
    }
    if (c == 0 && warp == NRW && lane < NB_TILE) {  // the least squares as the cycle's start left it
        const KState* ks = a.ks + r0 + lane;
        for (int i = 0; i <= MSMAX; ++i) S.g[lane][i] = ks->g[i];
        S.tol[lane] = ks->tol_abs;
    }
    __syncthreads();
    // The push of step jh - 1 (warp NRW of chunk 0) runs while the other warps
    // apply A for step jh to every right-hand side that took step jh - 1: its
    // stop decisions are read after the first barrier, and a right-hand side that
    // stopped at jh - 1 leaves its speculative phase-1 values unused (they go to
    // basis row jh + 1 beyond its last column, and to partial slots nothing reads).
    unsigned spec = gate_mask(a.gbuf, r0, 0);  // right-hand sides taking step 0
    int jh = 0;
    for (; jh < ms && spec; ++jh) {
        const int* gate = a.gbuf + (jh & 1) * a.nbp;
        const bool spec_on = rw && ((spec >> rl) & 1u);
        // phase 1: w = A v_jh, partial sums of V^+ w (speculative for step jh > 0)
        if (rw) phase_apply_staged<F16>(a, jh, r0, s0, ns, spec, wsb, wst, S.abuf[warp], NRW);
        else if (jh > 0 && warp == NRW && c == 0 && lane < NB_TILE &&
                 __ldcg(a.gbuf + ((jh - 1) & 1) * a.nbp + r0 + lane) == jh - 1)
            push_cycle(a, S, lane, r0 + lane, jh - 1, S.hs[lane]);  // warp `lane` (part 0) holds h2
        __syncthreads();
        CB_STAMP(6);
        if (spec_on) CB_DISPATCH(jh, (phase_gram1<JB>(a, jh, r, slot, s0, ne, e0, es, wsb + rl * wst, S.red[warp])));
        CB_STAMP(0);
        tile_sync(bar, a.nchunks, spin, err);
        CB_STAMP(1);
        // the gates of step jh are now final (the same in every CTA of the tile, read
        // from L2, which every SM sees alike): all leave the loop together
        const unsigned live = gate_mask(gate, r0, jh);
        if (!live) break;
        const bool on = rw && ((live >> rl) & 1u);
        // phase 2: h1 (every warp adds the chunk partials in the same order), w -= V h1,
        // partial sums of V^+ w and ||w||^2
        if (on) {
            float2 t;
            CB_DISPATCH(jh, (t = chunk_totals<JB>(a.p1, nslot, r, jh, false, nullptr, S.red[warp])));
            if (lane <= jh) {
                S.hs[warp][lane] = t;
                if (c == 0 && part == 0) S.h1[rl][lane] = t;
            }
            __syncwarp();
            CB_DISPATCH(jh, (phase_update_gram<false, JB>(a, jh, r, slot, s0, ne, e0, es, S.hs[warp], S.red[warp])));
        }
        CB_STAMP(2);
        tile_sync(bar, a.nchunks, spin, err);
        CB_STAMP(3);
        // phase 3: h2 and h_{j+1,j}; v_{j+1} (its push comes with the next step)
        if (on) {
            float2 t;
            float nrm = 0.f;
            CB_DISPATCH(jh, (t = chunk_totals<JB>(a.p2, nslot, r, jh, true, &nrm, S.red[warp])));
            const float hn = subdiag(t, jh, nrm);
            if (lane <= jh) S.hs[warp][lane] = t;
            if (lane == 0 && part == 0) S.hn[rl] = hn;
            __syncwarp();
            CB_DISPATCH(jh, (phase_update<JB>(a, jh, r, s0, ne, e0, es, S.hs[warp], hn > 0.f ? 1.f / hn : 0.f)));
        }
        CB_STAMP(4);
        tile_sync(bar, a.nchunks, spin, err);
        CB_STAMP(5);
        spec = live;
#ifdef CB_PHASE_CLOCKS
        ++steps;
#endif
    }
    // the last step's push, when the loop ran to the cycle length (after an early
    // exit every push has run: the exit follows the phase that pushed)
    if (jh == ms && warp == NRW && c == 0 && lane < NB_TILE &&
        __ldcg(a.gbuf + ((ms - 1) & 1) * a.nbp + r0 + lane) == ms - 1)
        push_cycle(a, S, lane, r0 + lane, ms - 1, S.hs[lane]);
#ifdef CB_PHASE_CLOCKS
    if (clk && threadIdx.x == 0 && steps > 0)
        printf("cb_cycle phases (ns/step over %d steps, %d chunks): apply %llu, gram1 %llu, bar1 %llu, "
               "update+gram2 %llu, bar2 %llu, update %llu, bar3 %llu\n",
               steps, a.nchunks, acc_t[6] / steps, acc_t[0] / steps, acc_t[1] / steps, acc_t[2] / steps,
               acc_t[3] / steps, acc_t[4] / steps, acc_t[5] / steps);
#endif
}

__global__ void k_cb_gate_init(CBArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < a.nbp) {
        a.gbuf[r] = a.ks[r].step_gate;
        a.gbuf[a.nbp + r] = -1;  // no stale index of an earlier cycle can match a step
    }
}

}  // namespace

void cb_geometry(CBArgs& a, long nsite, int nbp) {
    const int ntiles = nbp / NB_TILE;
    // about four CTAs per SM over (chunks x tiles), at most CB_MAXSPC sites and
    // CB_MAXCH chunks
    long spc = (nsite * ntiles + 4L * sm_count() - 1) / (4L * sm_count());
    spc = std::max(spc, (nsite + CB_MAXCH - 1) / CB_MAXCH);
    spc = std::max(1L, std::min((long)CB_MAXSPC, spc));
    if ((nsite + spc - 1) / spc > CB_MAXCH) spc = (nsite + CB_MAXCH - 1) / CB_MAXCH;  // caller rejects spc > CB_MAXSPC
    a.spc = (int)spc;
    a.nchunks = (int)((nsite + spc - 1) / spc);
    a.nbp = nbp;
    a.coop = 0;
}

// dynamic shared memory of the cycle kernel for chunks of spc sites
size_t cb_cycle_smem(long spc) { return sizeof(CBCycleSmem) + (size_t)NB_TILE * spc * NDOF * sizeof(float2); }
// the most the device allows one CTA (opt-in), which bounds spc
int cb_cycle_smem_max() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                                                 cudaSuccess) {
        (void)cudaGetLastError();
        return (int)cb_cycle_smem(CB_MAXSPC);
    }
    return v;
}

// shared memory of every coarse block kernel, allowed once per device
mg_status cb_configure() {
    static bool done[64] = {};
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 0;
    if (done[dev]) return MG_OK;
    const int sm = (int)sizeof(CBSmem);
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_apply_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_apply_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_update_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_update_push, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    const int smc = cb_cycle_smem_max();
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_cycle<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_cb_cycle<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smc));
    done[dev] = true;
    return MG_OK;
}

namespace {
bool cb_geometry_cycle_uncached(CBArgs& a, long nsite, int nbp, bool fp16);
}

// cb_geometry_cycle_uncached per (device, coarse sites, block, format), computed
// once (its occupancy queries would otherwise cost host time every coarse solve)
bool cb_geometry_cycle(CBArgs& a, long nsite, int nbp, bool fp16) {
    struct Entry {
        int dev;
        long nsite;
        int nbp;
        bool fp16, ok;
        int spc, nchunks;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry& e : cache)
            if (e.dev == dev && e.nsite == nsite && e.nbp == nbp && e.fp16 == fp16) {
                if (!e.ok) return false;
                a.spc = e.spc;
                a.nchunks = e.nchunks;
                a.nbp = nbp;
                a.coop = 1;
                return true;
            }
    }
    const bool ok = cb_geometry_cycle_uncached(a, nsite, nbp, fp16);
    std::lock_guard<std::mutex> lock(mu);
    cache.push_back(Entry{dev, nsite, nbp, fp16, ok, ok ? a.spc : 0, ok ? a.nchunks : 0});
    return ok;
}

namespace {
bool cb_geometry_cycle_uncached(CBArgs& a, long nsite, int nbp, bool fp16) {
    const int ntiles = nbp / NB_TILE;
    if (cb_configure() != MG_OK) return false;
    const size_t smax = (size_t)cb_cycle_smem_max();
    // the fewest sites per chunk whose grid is resident at once; the shared memory
    // of w grows with the chunk, so the resident count is queried per candidate
    for (long spc = std::max(1L, (nsite * ntiles + (long)sm_count() * 4 - 1) / ((long)sm_count() * 4)); spc <= nsite;
         ++spc) {
        const size_t sm = cb_cycle_smem(spc);
        if (sm > smax) return false;
        const long nch = (nsite + spc - 1) / spc;
        if (nch * CB_WPR > CB_MAXCH) continue;
        int per_sm = 0;
        cudaError_t e = fp16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cb_cycle<true>, CB_COOP_THREADS, sm)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cb_cycle<false>, CB_COOP_THREADS, sm);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        if (per_sm < 1 || nch * ntiles > (long)per_sm * sm_count()) continue;
        a.spc = (int)spc;
        a.nchunks = (int)nch;
        a.nbp = nbp;
        a.coop = 1;
        return true;
    }
    return false;
}
}  // namespace

void launch_cb_gate_init(const CBArgs& a, cudaStream_t s) {
    k_cb_gate_init<<<(a.nbp + 63) / 64, 64, 0, s>>>(a);
    count_launch();
}

void launch_cb_step(const CBArgs& a, int jh, bool fp16, cudaStream_t s) {
    if (cb_configure() != MG_OK) return;
    const dim3 grid(a.nchunks, a.nbp / NB_TILE);
    const size_t sm = sizeof(CBSmem);
    if (fp16) k_cb_apply_gram<true><<<grid, CB_THREADS, sm, s>>>(a, jh);
    else k_cb_apply_gram<false><<<grid, CB_THREADS, sm, s>>>(a, jh);
    k_cb_update_gram<<<grid, CB_THREADS, sm, s>>>(a, jh);
    k_cb_update_push<<<grid, CB_THREADS, sm, s>>>(a, jh);
    count_launch(3);
}

mg_status launch_cb_cycle(const CBArgs& a, int ms, bool fp16, long spin, int* err, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    MG_TRY(cb_configure());
    cfg.gridDim = dim3(a.nchunks, a.nbp / NB_TILE);
    cfg.blockDim = dim3(CB_COOP_THREADS);
    cfg.dynamicSmemBytes = cb_cycle_smem(a.spc);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (fp16) MG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cb_cycle<true>, a, ms, spin, err));
    else MG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cb_cycle<false>, a, ms, spin, err));
    count_launch();
    return MG_OK;
}

}  // namespace mg
