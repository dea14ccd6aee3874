// The whole GMRES-Proj(m,k) coarsest-grid solve (Section 2; Morgan & Wilcox)
// in one thread-block-cluster kernel.
//
// The coarsest grid is small (256 sites x 24 dofs at 256^2) and its solve runs
// ~10^3 Krylov steps per outer iteration, so a step is bound by latency, not
// by bytes.  One cluster of up to 16 CTAs runs a whole solve: reductions
// through distributed shared memory, and the small least-squares work done
// redundantly (and identically) by every CTA, so no CTA ever waits for another
// one's scalar result.  Several solves (one per stream) run side by side on
// different clusters.
//
// Work split: CTA b of the cluster owns sites [b*spc, (b+1)*spc) and their 24
// dofs.  When it fits, the CTA keeps its rows of the Krylov basis in shared
// memory, so the Gram and update passes never leave the SM (the deflation
// space, read once per cycle, stays in global memory).  Each new basis row is
// then pushed straight into the staging slots of the five sites whose apply
// reads it (push mode, other CTAs' slots by distributed shared-memory stores).
// Otherwise the basis goes through global memory (L2-resident), from where the
// apply stages the five neighbour rows of each own site.  Neighbour and push
// tables are built once per launch.
//
// Per Arnoldi step j (CGS2, as in the rest of the library):
//   w = A v_j; h1 = V^+ w: partials pushed to every CTA          [exchange]
//   reduce h1; w -= V h1; h2 = V^+ w, n2 = ||w||^2: pushed        [exchange]
//   reduce; h_{j+1,j} = sqrt(n2 - |h2|^2) (V orthonormal);
//   v_{j+1} = (w - V h2) / h_{j+1,j}, pushed to the staging slots [exchange]
//   Givens update of the least squares and the residual estimate
// In push mode an exchange is dataflow: the values go by st.async into the
// receivers' shared memory, counted in bytes on an mbarrier there, and an extra
// least-squares warp runs the Givens update of step j during the apply of step
// j + 1.  Otherwise an exchange is a hardware cluster barrier after plain
// distributed shared-memory stores (the last one split, with warp 0's Givens
// update between its arrive and wait).  Reductions add the CTAs' partials in
// rank order with one fixed warp tree, so every CTA holds bit-identical scalars
// and takes identical control decisions, and each reduction reads only local
// shared memory.
//
// The small least squares runs in the precision of the vectors (FP32 in the
// mixed-precision V-cycle, FP64 on the plain path).
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "coarse_coop.cuh"

namespace cg = cooperative_groups;

namespace mg {

namespace {

constexpr int NDOF = 24;
constexpr int MAX_THREADS = 512;
constexpr int MAX_SPC = 16;       // sites per apply chunk (staged neighbour rows)
constexpr int MAX_NB_SITES = 64;  // sites per CTA in the neighbour table
constexpr int MAX_CLUSTER = 16;    // CTAs of one cluster (non-portable size)
constexpr size_t SMEM_LIMIT = 227 * 1024;
constexpr long FLOW_SPIN = 1L << 20;  // default try_wait rounds before a dataflow wait gives up
// FP16 operator (push mode): the blocks of directions 0..ASH_DIRS-1 of a CTA's
// sites stay in its shared memory for the whole solve, the other directions
// stream from L2 each step.  A site's part is padded by 24 words so that the two
// sites one warp reads fall on different banks.
constexpr int ASH_DIRS = 3;
constexpr int ASH_SITE_WORDS = ASH_DIRS * 24 * 24 + 24;

template <typename R>
struct Small {  // per-CTA copy of the small least-squares state, precision R
    using Z = C2<R>;
    Z H[(MSMAX + 1) * MSMAX];  // column-major, ld MSMAX + 1 (unrotated)
    Z Rm[(MSMAX + 1) * MSMAX];
    R rc[MSMAX];
    Z rs[MSMAX];
    Z g[MSMAX + 1], c[MSMAX + 1], d[MSMAX], rho[MSMAX + 1];
    Z pd[KMAX], pu[KLD];       // projection coefficients
};

template <typename T>
struct ClusterSmem {
    // partial sums and reduced values in the vectors' precision: FP64 adds run at
    // a small fraction of the FP32 rate on this GPU, and the reductions sit on the
    // critical path of every Arnoldi step
    C2<T> inbox[2][MAX_CLUSTER][PSTR];   // partial sums pushed here by every CTA of the cluster
    C2<T> red[PSTR];                     // reduced values (identical in every CTA)
    C2<T> h1[MSMAX + 1];
    C2<T> xs[MAX_SPC][5][NDOF];          // staged neighbour rows
    int nbt[MAX_NB_SITES][5];            // neighbour site of each own site and direction
    int pusht[MAX_SPC][5];               // where each own row goes: (CTA, site, direction) of xs
    Small<T> st;
    T scal[8];
    int ctl[8];
    unsigned long long mb[4];  // dataflow mode: arrivals of inbox[0], inbox[1] and xs; [3]: the
                               // probe's barrier, which nothing completes
    int fault;                 // dataflow mode: a wait gave up
    int fpub[2];               // fault as published at a cycle's first cluster barrier (by cycle parity)
    C2<T> zc[MSMAX + 1];       // delayed CGS2: coefficients of the u_{j+1} update
    C2<T> hnext[MSMAX + 1];    // delayed CGS2: first projection of A q_j
};

// dynamic shared memory: ClusterSmem, then (optionally) the basis slice
// Vs[(ms + 1)][rows], then the projection matrices M (k x (k+1)) and
// N ((k+1) x (k+1)), both column-major
template <typename T>
__host__ __device__ inline size_t slice_bytes(int ms, int rows) {
    return (size_t)(ms + 1) * rows * sizeof(C2<T>);
}
template <typename T>
__host__ __device__ inline size_t proj_bytes(int k) {
    return (size_t)(k * (k + 1) + (k + 1) * (k + 1)) * sizeof(C2<T>);
}

template <typename R>
__device__ __forceinline__ R cabs_(C2<R> a) { return sqrt(a.x * a.x + a.y * a.y); }

template <typename R>
__device__ __forceinline__ C2<R> cdiv_(C2<R> a, C2<R> b) {
    if (fabs(b.x) >= fabs(b.y)) {
        R r = b.y / b.x, den = b.x + b.y * r;
        return mk<R>((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    R r = b.x / b.y, den = b.x * r + b.y;
    return mk<R>((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// acc - a * b with every rounding step fixed: both cluster kernels get the same
// operations, whatever contraction the compiler would pick for a * b - c * d
template <typename R>
__device__ __forceinline__ C2<R> cfms_(C2<R> a, C2<R> b, C2<R> acc) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// d = R^{-1} g for the jc x jc upper-triangular R (column-major, leading
// dimension MSMAX + 1, jc <= MSMAX < 32) by one warp, column by column. The
// lanes first form the reciprocals of their pivots at once (a zero pivot gives
// zero, so d_i = 0 there); then lane i keeps g_i minus the columns already
// eliminated, and in turn i its d_i = (that) / R_ii is broadcast to the lanes
// above.  Only a product, a shuffle and a subtraction stay on the serial chain.
template <typename R>
__device__ __forceinline__ void back_subst_warp(const C2<R>* Rm, const C2<R>* g, C2<R>* d, int jc, int lane) {
    constexpr int LDR = MSMAX + 1;
    C2<R> inv = mk<R>(0, 0), acc = mk<R>(0, 0);
    if (lane < jc) {
        const C2<R> piv = Rm[lane + LDR * lane];
        if (piv.x != R(0) || piv.y != R(0)) inv = cdiv_<R>(mk<R>(1, 0), piv);
        acc = g[lane];
    }
    for (int i = jc - 1; i >= 0; --i) {
        const C2<R> rli = (lane < i) ? Rm[lane + LDR * i] : mk<R>(0, 0);
        C2<R> di = mk<R>(fma(-acc.y, inv.y, acc.x * inv.x), fma(acc.y, inv.x, acc.x * inv.y));
        di.x = __shfl_sync(0xffffffffu, di.x, i);
        di.y = __shfl_sync(0xffffffffu, di.y, i);
        if (lane == i) d[i] = di;
        if (lane < i) acc = cfms_<R>(rli, di, acc);
    }
}

template <typename R>
__device__ __forceinline__ R rsqrt_(R x) {
    if constexpr (std::is_same<R, float>::value)
        return rsqrtf(x);
    else
        return rsqrt(x);
}

// Complex Givens rotation G = [[c, s], [-conj(s), c]] with G [a; h] = [r; 0]
// for a real, non-negative h (the new subdiagonal entry).
template <typename R>
__device__ __forceinline__ void givens_real_(C2<R> a, R h, R& c, C2<R>& s, C2<R>& r) {
    if (h == R(0)) { c = R(1); s = mk<R>(0, 0); r = a; return; }
    const R aa2 = a.x * a.x + a.y * a.y;
    if (aa2 == R(0)) { c = R(0); s = mk<R>(1, 0); r = mk<R>(h, 0); return; }
    // reciprocal square roots only: no divide on this serial path
    const R rh2 = aa2 + h * h;
    const R inv_aa = rsqrt_(aa2), inv_rh = rsqrt_(rh2);
    c = aa2 * inv_aa * inv_rh;
    const C2<R> ph = mk<R>(a.x * inv_aa, a.y * inv_aa);
    s = cscale(ph, h * inv_rh);
    r = cscale(ph, rh2 * inv_rh);
}
template <typename R>
__device__ __forceinline__ void rot_(R c, C2<R> s, C2<R>& up, C2<R>& uq) {
    const C2<R> p = up, q = uq;
    up = cadd(cscale(p, c), cmul(s, q));
    uq = csub(cscale(q, c), cmul(conj_(s), p));
}

// One complex entry of the FP16 operator copy (real part in the low half)
template <typename T>
__device__ __forceinline__ C2<T> half_bits(unsigned u) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
    return mk<T>((T)f.x, (T)f.y);
}
template <typename T>
__device__ __forceinline__ C2<T> half_entry(const unsigned* p) {
    return half_bits<T>(__ldg(p));
}

// ---- tensor-core apply of the FP16 operator (a.mma) ----
// The staged vector holds each complex entry x as two FP16 pairs: hi = (Re, Im)
// of x 2^10 rounded to FP16, lo = the same of the remainder, in the two words of
// one 8-byte slot.  2^10 keeps both parts normal for the entries of a unit
// vector and leaves a factor 64 below the FP16 range; hi + lo carries 22 bits.
constexpr float TC_XS = 1024.f;
constexpr float TC_XS_INV = 1.f / 1024.f;

__device__ __forceinline__ float2 tc_split(float2 v) {
    const __half2 hi = __floats2half2_rn(v.x * TC_XS, v.y * TC_XS);
    const float2 hf = __half22float2(hi);
    // v 2^10 - hi is exact in FP32 (hi is v 2^10 rounded to 11 bits)
    const __half2 lo = __floats2half2_rn(fmaf(v.x, TC_XS, -hf.x), fmaf(v.y, TC_XS, -hf.y));
    return make_float2(__uint_as_float(*reinterpret_cast<const unsigned*>(&hi)),
                       __uint_as_float(*reinterpret_cast<const unsigned*>(&lo)));
}
template <typename T>
__device__ __forceinline__ C2<T> stage_value(C2<T> v, bool split) {
    if constexpr (std::is_same<T, float>::value) return split ? tc_split(v) : v;
    return v;
}

// Word of the B fragment that lane column n = g (0..7) takes from a staged entry
// p (rows 2l, 2l + 1 of the real form): n = 0: (Re hi, -Im hi), 1: (Im hi, Re hi),
// 2 and 3: the same of lo, 4..7: zero.  The low half is the lower row.
__device__ __forceinline__ unsigned tc_bword(float2 p, int g) {
    const unsigned src = __float_as_uint((g & 2) ? p.y : p.x);
    const unsigned w = (g & 1) ? __byte_perm(src, 0u, 0x1032) : (src ^ 0x80000000u);
    return g < 4 ? w : 0u;
}

__device__ __forceinline__ void tc_mma(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                       unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// w = sum_d A_d x_d for one own site on tensor cores (m16n8k16, FP16 inputs,
// FP32 accumulation), by one whole warp.  Each complex product is the real
// product A'' B'': A'' (24 x 48) has Re and Im of column l of A_d in columns
// 2l and 2l + 1, so a stored FP16 word (real part in the low half) is already
// an element pair of an A fragment; B'' (48 x 8) holds in rows 2l, 2l + 1 the
// pairs of tc_bword for the staged x_d[l].  Then Re w = (column 0 + column 2)
// 2^-10 and Im w = (column 1 + column 3) 2^-10.  The 24 rows are two M tiles,
// the second with rows 24..31 zero; the 5 directions x 24 columns are 15 K
// tiles.  Blocks are column-major: entry (row i, column l) of direction d is
// word (d 24 + l) 24 + i.  Directions < ASH_DIRS come from shared memory, the
// others from the FP16 operator in global memory, whose fragments
// (tc_load_stream) are loaded first, so that their latency overlaps the
// shared-memory directions, which every site accumulates first.
constexpr int TC_SW = (5 - ASH_DIRS) * 3 * 6;  // stream fragment words a lane holds for one site
struct TcAcc {
    float m0[4], m1[4];  // M tiles 0 (rows 0..15) and 1 (rows 16..23)
};
__device__ __forceinline__ void tc_zero(TcAcc& c) {
#pragma unroll
    for (int u = 0; u < 4; ++u) c.m0[u] = c.m1[u] = 0.f;
}
// the A fragments of direction d, K tile kt from a site's blocks p (lane offset applied)
__device__ __forceinline__ void tc_frag(const unsigned* p, unsigned (&q)[6]) {
    q[0] = p[0];
    q[1] = p[8];
    q[2] = p[4 * NDOF];
    q[3] = p[4 * NDOF + 8];
    q[4] = p[16];
    q[5] = p[4 * NDOF + 16];
}
__device__ __forceinline__ void tc_step(TcAcc& c, const unsigned (&q)[6], float2 x0, float2 x1, int g) {
    const unsigned b0 = tc_bword(x0, g), b1 = tc_bword(x1, g);
    tc_mma(c.m0, q[0], q[1], q[2], q[3], b0, b1);
    tc_mma(c.m1, q[4], 0u, q[5], 0u, b0, b1);
}
// fragments of the streamed directions of one site (Ag: the site's blocks)
__device__ __forceinline__ void tc_load_stream(const unsigned* __restrict__ Ag, unsigned (&f)[TC_SW], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int d = ASH_DIRS; d < 5; ++d)
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            const unsigned* p = Ag + (d * NDOF + 8 * kt + t) * NDOF + g;
            unsigned* q = f + ((d - ASH_DIRS) * 3 + kt) * 6;
            q[0] = __ldg(p);
            q[1] = __ldg(p + 8);
            q[2] = __ldg(p + 4 * NDOF);
            q[3] = __ldg(p + 4 * NDOF + 8);
            q[4] = __ldg(p + 16);
            q[5] = __ldg(p + 4 * NDOF + 16);
        }
}
__device__ __forceinline__ void tc_stream_dirs(TcAcc& c, const unsigned (&f)[TC_SW], const float2 (*xs)[NDOF],
                                               int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int d = ASH_DIRS; d < 5; ++d)
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            unsigned q[6];
#pragma unroll
            for (int u = 0; u < 6; ++u) q[u] = f[((d - ASH_DIRS) * 3 + kt) * 6 + u];
            tc_step(c, q, xs[d][8 * kt + t], xs[d][8 * kt + t + 4], g);
        }
}
// As: the site's shared-memory blocks
__device__ __forceinline__ void tc_shared_dirs(TcAcc& c, const unsigned* As, const float2 (*xs)[NDOF], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int d = 0; d < ASH_DIRS; ++d)
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            unsigned q[6];
            tc_frag(As + (d * NDOF + 8 * kt + t) * NDOF + g, q);
            tc_step(c, q, xs[d][8 * kt + t], xs[d][8 * kt + t + 4], g);
        }
}
// out[0..23] = c 2^-10: lane t = 0 holds columns 0, 1 (hi) and lane t = 1
// columns 2, 3 (lo) of rows g, g + 8 (M tile 0) and 16 + g (M tile 1)
__device__ __forceinline__ void tc_store(const TcAcc& c, float2* out, int lane) {
    const int g = lane >> 2, t = lane & 3;
    float r[6] = {c.m0[0], c.m0[1], c.m0[2], c.m0[3], c.m1[0], c.m1[1]};
#pragma unroll
    for (int u = 0; u < 6; ++u) r[u] += __shfl_xor_sync(0xffffffffu, r[u], 1);
    if (t == 0) {
        out[g] = make_float2(r[0] * TC_XS_INV, r[1] * TC_XS_INV);
        out[g + 8] = make_float2(r[2] * TC_XS_INV, r[3] * TC_XS_INV);
        out[g + 16] = make_float2(r[4] * TC_XS_INV, r[5] * TC_XS_INV);
    }
}

// Store v at the address dst has in the shared memory of CTA `rank` of the
// cluster (a plain shared-memory store when rank == me).
template <typename T>
__device__ __forceinline__ void st_rank(C2<T>* dst, int rank, int me, C2<T> v) {
    if (rank == me) {
        *dst = v;
        return;
    }
    const unsigned la = (unsigned)__cvta_generic_to_shared(dst);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(la), "r"(rank));
    if constexpr (std::is_same<T, float>::value)
        asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(ra), "f"(v.x), "f"(v.y) : "memory");
    else
        asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};\n" ::"r"(ra), "d"(v.x), "d"(v.y) : "memory");
}

// Partials of nd inner products conj(X[i]) . y over the CTA's rows (X, y point
// at the own rows; warp per product, lanes over rows), plus optionally ||y||^2
// in slot nd.  Each partial is pushed into every CTA's inbox (row = this CTA's
// rank), so after the next cluster barrier every CTA reduces from its own
// shared memory instead of fetching from 16 remote ones.
template <typename T>
__device__ void push_gram(cg::cluster_group& cluster, const C2<T>* X, long ldx, int nd, const C2<T>* y, int nrows,
                          bool norm, C2<T>* inbox, int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp >= nw) return;  // the least-squares warp takes no products
    const int nr = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
    const int ntot = nd + (norm ? 1 : 0);
    for (int i = warp; i < ntot; i += nw) {
        // four independent accumulators keep four loads per lane in flight
        C2<T> acc4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc4[u] = mk<T>(0, 0);
        const C2<T>* xi = (i < nd) ? X + (long)i * ldx : y;
        int e = lane;
        for (; e + 96 < nrows; e += 128) {
            C2<T> xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xv[u] = xi[e + 32 * u];
                yv[u] = y[e + 32 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc4[u] = cfmac(xv[u], yv[u], acc4[u]);
        }
        for (; e < nrows; e += 32) acc4[0] = cfmac(xi[e], y[e], acc4[0]);
        C2<T> acc = cadd(cadd(acc4[0], acc4[1]), cadd(acc4[2], acc4[3]));
        if (i >= nd) acc.y = 0;  // ||y||^2 = conj(y) . y is real
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane < nr) *cluster.map_shared_rank(inbox + me * PSTR + i, lane) = acc;
    }
}

// acc +/- sum_{i < cnt} X[i][e] coef[i], loading eight rows of X at a time
template <typename T, bool SUB>
__device__ __forceinline__ C2<T> accum_rows(C2<T> acc, const C2<T>* X, long ldx, int e, const C2<T>* coef,
                                            int cnt) {
    int i = 0;
    for (; i + 8 <= cnt; i += 8) {
        C2<T> v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = X[(long)(i + u) * ldx + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = SUB ? cfms_<T>(v[u], coef[i + u], acc) : cfma(v[u], coef[i + u], acc);
    }
    for (; i < cnt; ++i) {
        const C2<T> v = X[(long)i * ldx + e];
        acc = SUB ? cfms_<T>(v, coef[i], acc) : cfma(v, coef[i], acc);
    }
    return acc;
}

// accum_rows for two right-hand sides at once (their loads interleaved; per
// right-hand side the order of accum_rows)
template <typename T, bool SUB>
__device__ __forceinline__ void accum_rows2(C2<T>& acc0, C2<T>& acc1, const C2<T>* X0, const C2<T>* X1, long ldx,
                                            int e, const C2<T>* coef0, const C2<T>* coef1, int cnt) {
    int i = 0;
    for (; i + 8 <= cnt; i += 8) {
        C2<T> v[8], w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            v[u] = X0[(long)(i + u) * ldx + e];
            w[u] = X1[(long)(i + u) * ldx + e];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc0 = SUB ? cfms_<T>(v[u], coef0[i + u], acc0) : cfma(v[u], coef0[i + u], acc0);
            acc1 = SUB ? cfms_<T>(w[u], coef1[i + u], acc1) : cfma(w[u], coef1[i + u], acc1);
        }
    }
    for (; i < cnt; ++i) {
        const C2<T> v = X0[(long)i * ldx + e], w = X1[(long)i * ldx + e];
        acc0 = SUB ? cfms_<T>(v, coef0[i], acc0) : cfma(v, coef0[i], acc0);
        acc1 = SUB ? cfms_<T>(w, coef1[i], acc1) : cfma(w, coef1[i], acc1);
    }
}

// Sum the pushed partials of all CTAs of the cluster in rank order (every CTA
// gets the same result): red[i] = sum_r inbox[r][i], i < n.  Called once all
// partials are in: after the cluster barrier, or the dataflow wait, that
// follows the pushes.
template <typename T>
__device__ void reduce_inbox(const C2<T>* inbox, int nr, int n, C2<T>* red, int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n && warp < nw; i += nw) {
        C2<T> a = mk<T>(0, 0);
        if (lane < nr) a = inbox[lane * PSTR + i];
        // at most MAX_CLUSTER = 16 partials: lanes 16..31 hold zeros
#pragma unroll
        for (int o = MAX_CLUSTER / 2; o > 0; o >>= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        }
        if (lane == 0) red[i] = a;
    }
    __syncthreads();
}

// Split cluster barrier: arrive (releasing this thread's writes, shared and
// global, to the cluster) and wait (acquiring everyone's).  Work placed between
// the two overlaps the barrier's latency.  Every thread of a warp executes both.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Dataflow exchange (push mode): instead of a cluster barrier after each push,
// every value goes out by st.async, which counts its bytes on an mbarrier in the
// receiving CTA; a CTA goes on once its barrier has seen all the bytes of the
// phase (armed by its thread 0 with the expected count).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_addr(unsigned local, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait for the completion of the phase with this parity (acquiring the
// cluster's st.async writes); false when it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long spin) {
    const unsigned addr = smem_addr(bar);
    for (long it = 0; it < spin; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// barrier 1 over the first nthreads threads (the row warps)
__device__ __forceinline__ void row_warps_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ void st_async(unsigned dst, float2 v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(dst),
                 "f"(v.x), "f"(v.y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async(unsigned dst, double2 v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];\n" ::"r"(dst),
                 "d"(v.x), "d"(v.y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ long nbr_site(long s, int d, int Nx, int Nt) {
    const int xx = (int)(s % Nx), tt = (int)(s / Nx);
    if (d == 1) return (xx + 1 == Nx) ? s - xx : s + 1;
    if (d == 2) return (xx == 0) ? s + Nx - 1 : s - 1;
    if (d == 3) return (tt + 1 == Nt) ? (long)xx : s + Nx;
    if (d == 4) return (tt == 0) ? s + (long)Nx * (Nt - 1) : s - Nx;
    return s;
}

// Write element k of own row (site ls) of a new basis vector into the five
// staging slots that read it (push mode); split: as the tensor-core apply's
// two FP16 parts (tc_split).
template <typename T>
__device__ __forceinline__ void push_row(ClusterSmem<T>& S, int me, int e, C2<T> v, bool split) {
    const int ls = e / NDOF, kk = e - ls * NDOF;
    const C2<T> sv = stage_value<T>(v, split);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int code = S.pusht[ls][q];
        st_rank<T>(&S.xs[(code >> 3) & 0x1fff][code & 7][kk], code >> 16, me, sv);
    }
}

// push_gram and push_row in dataflow mode: the same values to the same places,
// by st.async counted on the receiver's barrier bar (inbox or staging slots).
template <typename T>
__device__ void push_gram_flow(const C2<T>* X, long ldx, int nd, const C2<T>* y, int nrows, bool norm, C2<T>* inbox,
                               unsigned long long* bar, int nr, int me, int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp >= nw) return;
    const int ntot = nd + (norm ? 1 : 0);
    const unsigned bar_r = lane < nr ? cluster_addr(smem_addr(bar), lane) : 0u;
    for (int i = warp; i < ntot; i += nw) {
        C2<T> acc4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc4[u] = mk<T>(0, 0);
        const C2<T>* xi = (i < nd) ? X + (long)i * ldx : y;
        int e = lane;
        for (; e + 96 < nrows; e += 128) {
            C2<T> xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xv[u] = xi[e + 32 * u];
                yv[u] = y[e + 32 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc4[u] = cfmac(xv[u], yv[u], acc4[u]);
        }
        for (; e < nrows; e += 32) acc4[0] = cfmac(xi[e], y[e], acc4[0]);
        C2<T> acc = cadd(cadd(acc4[0], acc4[1]), cadd(acc4[2], acc4[3]));
        if (i >= nd) acc.y = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane < nr) st_async(cluster_addr(smem_addr(inbox + me * PSTR + i), lane), acc, bar_r);
    }
}
template <typename T>
__device__ __forceinline__ void push_row_flow(ClusterSmem<T>& S, int e, C2<T> v, bool split) {
    const int ls = e / NDOF, kk = e - ls * NDOF;
    const unsigned bar = smem_addr(&S.mb[2]);
    const C2<T> sv = stage_value<T>(v, split);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int code = S.pusht[ls][q], owner = code >> 16;
        st_async(cluster_addr(smem_addr(&S.xs[(code >> 3) & 0x1fff][code & 7][kk]), owner), sv,
                 cluster_addr(bar, owner));
    }
}

#ifdef CP_PHASE_CLOCKS
// phase timing of thread 0 of CTA 0 (a build with -DCP_PHASE_CLOCKS): the cycles
// of each phase of the dataflow Arnoldi step, averaged per launch and printed
// for the first launches
__device__ unsigned cp_clock_launches = 0;
#define CP_STAMP(k)                              \
    do {                                         \
        if (clk) {                               \
            const long long now = clock64();     \
            acc_t[k] += now - t_prev;            \
            t_prev = now;                        \
        }                                        \
    } while (0)
#else
#define CP_STAMP(k) \
    do {            \
    } while (0)
#endif

// At most 128 registers a thread, so that a CTA of up to 512 threads fits one
// SM (512 x 128 = 65536).  A solve is latency-bound; the registers go to more
// operator loads in flight in the apply, which was measured faster, also with
// ten concurrent solves, than fitting two CTAs per SM with 80 registers.
template <typename T>
__global__ void __maxnreg__(128) k_coarse_proj(CoopArgs<T> a) {
    using Z = C2<T>;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ClusterSmem<T>& S = *reinterpret_cast<ClusterSmem<T>*>(smem_raw);
    Small<T>& st = S.st;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rank = (int)cluster.block_rank();
    const long nsite = (long)a.Nx * a.Nt;
    const long n = nsite * NDOF;
    const long s0 = (long)rank * a.spc;
    const long s1 = min(nsite, s0 + a.spc);
    const int my_sites = (int)max(0L, s1 - s0);
    const long r0 = s0 * NDOF;
    const int nrows = my_sites * NDOF;
    const int k = a.k, ms = a.ms;
    const int LD = MSMAX + 1;
    // with a.lsw the last warp owns no rows: it runs the least-squares update of
    // step j while the other (row) warps already apply A for step j + 1
    const int nwr = (int)(blockDim.x >> 5) - (a.lsw ? 1 : 0);
    const bool ls_warp = a.lsw && (tid >> 5) == nwr;
    const bool table = my_sites <= MAX_NB_SITES;

    // own rows of the basis: shared memory when it fits (the deflation space is
    // read once per cycle and stays in global memory)
    Z* Vl;
    const Z* Wl = a.W + r0;
    const long ldw = n;
    long ldv;
    if (a.vs) {
        Vl = reinterpret_cast<Z*>(smem_raw + sizeof(ClusterSmem<T>));
        ldv = a.spc * NDOF;
    } else {
        Vl = a.V + r0;
        ldv = n;
    }
    if (table)
        for (int e = tid; e < my_sites * 5; e += nt) S.nbt[e / 5][e % 5] = (int)nbr_site(s0 + e / 5, e % 5, a.Nx, a.Nt);
    // Push mode (the basis slice in shared memory and every CTA's sites in one
    // staging chunk): each new basis row is written straight into the staging
    // slots xs of the five sites that read it (self, -x, +x, -t, +t neighbours;
    // other CTAs' through distributed shared memory), so the apply after the
    // next barrier reads only local shared memory and the basis never goes
    // through global memory.  Slot q of own site u: the site w whose xs[w][d]
    // holds v(u), i.e. u = nbr(w, d).
    const bool push = a.vs && a.spc <= MAX_SPC;
    // dataflow mode (push mode with a.flow): the reductions of each Arnoldi step
    // and the staging of v_{j+1} go by st.async into barriers counted in bytes,
    // with no cluster barrier in the step.  Buffer reuse stays safe without one:
    // a CTA can send into a phase's inbox (or staging slots) only after it has
    // received this CTA's contribution to a later exchange, which this CTA makes
    // after it has read the buffer.
    const bool flow = push && a.flow;
    // tensor-core apply (tc_apply_site): FP32 dataflow mode with the FP16 operator,
    // its first directions in shared memory, and CGS2; the staging slots then hold
    // split values
    const bool mma = std::is_same<T, float>::value && flow && a.ash && a.mma && !a.dc;
#ifdef CP_PHASE_CLOCKS
    const bool clk = rank == 0 && tid == 0 && atomicAdd(&cp_clock_launches, 1u) < 48u;
    long long acc_t[7] = {0, 0, 0, 0, 0, 0, 0}, t_prev = clock64();
    int clk_steps = 0;
#endif
    const long spin = a.spin > 0 ? a.spin : FLOW_SPIN;
    unsigned fph[3] = {0u, 0u, 0u};  // parity of the next phase of each barrier (row warps)
    // A wait that gives up marks the CTA faulted.  From then on the CTA skips
    // its waits and stops arming its barriers (a phase is never armed twice
    // while incomplete; bytes that still arrive only lower the transaction
    // count of a phase nobody waits for), and at the next cycle's first cluster
    // barrier every CTA sees the fault and leaves the solve loop together.
    auto flow_wait = [&](int b) {
        if (!S.fault && !mbar_wait(&S.mb[b], fph[b], spin)) S.fault = 1;
        fph[b] ^= 1u;
    };
    auto arm = [&](int b, unsigned bytes) {
        if (tid == 0 && !S.fault) mbar_arm(&S.mb[b], bytes);
    };
    if (tid == 0) {
        if (flow) {
            for (int b = 0; b < 4; ++b) mbar_init(&S.mb[b], 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        S.fault = 0;
        S.fpub[0] = S.fpub[1] = 0;
    }
    if (push)
        for (int e = tid; e < my_sites * 5; e += nt) {
            const int ls = e / 5, q = e - ls * 5;
            const long u = s0 + ls;
            const int from[5] = {0, 2, 1, 4, 3};  // w = nbr(u, from[q]), d = q
            const long w = nbr_site(u, from[q], a.Nx, a.Nt);
            const int owner = (int)(w / a.spc);
            S.pusht[ls][q] = (owner << 16) | ((int)(w - (long)owner * a.spc) << 3) | q;
        }

    // Projection onto the deflation space, d = argmin ||W^+ r - H_k d||, as two
    // small matrices fixed for the whole solve: d = M g and H_k d = N g with
    // g = W^+ r, M = R^{-1} Q^+ from the QR factorisation of H_k (the stored
    // rotations and R), N = H_k M.  Warp 0 builds column l of both by solving
    // for g = e_l.
    Z* Mp = reinterpret_cast<Z*>(smem_raw + sizeof(ClusterSmem<T>) +
                                 (a.vs ? slice_bytes<T>(ms, a.spc * NDOF) : 0));
    Z* Np = Mp + k * (k + 1);
    if (tid < 32) {
        const KState* P = a.pls;
        for (int l = tid; l <= k; l += 32) {
            Z g[KLD], dd[KMAX];
            for (int i = 0; i <= k; ++i) g[i] = mk<T>(i == l ? T(1) : T(0), 0);
            for (int t = 0; t < P->nrot; ++t)
                rot_<T>((T)P->rc[t], from_d2<T>(P->rs[t]), g[P->ra[t]], g[P->rb[t]]);
            for (int i = k - 1; i >= 0; --i) {
                Z acc = g[i];
                for (int m = i + 1; m < k; ++m) acc = cfms_<T>(from_d2<T>(P->R[i + KLD * m]), dd[m], acc);
                dd[i] = cdiv_<T>(acc, from_d2<T>(P->R[i + KLD * i]));
            }
            for (int i = 0; i < k; ++i) Mp[i + k * l] = dd[i];
            for (int i = 0; i <= k; ++i) {
                Z acc = mk<T>(0, 0);
                for (int m = 0; m < k; ++m) acc = cfma(from_d2<T>(P->H[i + KLD * m]), dd[m], acc);
                Np[i + (k + 1) * l] = acc;
            }
        }
    }

    // a.ash: the FP16 blocks of the first ASH_DIRS directions of the own sites,
    // copied once into shared memory after M and N
    unsigned* Ash = reinterpret_cast<unsigned*>(Np + (k + 1) * (k + 1));
    if (a.ash)
        for (int e = tid; e < my_sites * ASH_DIRS * NDOF * NDOF; e += nt) {
            const int ls = e / (ASH_DIRS * NDOF * NDOF), q = e - ls * (ASH_DIRS * NDOF * NDOF);
            Ash[ls * ASH_SITE_WORDS + q] = a.Ah[(s0 + ls) * (5L * NDOF * NDOF) + q];
        }

    Z* xl = a.x + r0;
    Z* rl = a.r + r0;
    // x = 0, r = f, ||f||^2
    for (int e = tid; e < nrows; e += nt) {
        xl[e] = mk<T>(0, 0);
        rl[e] = a.f[r0 + e];
    }
    __syncthreads();
    const int ncta = (int)cluster.num_blocks();
    push_gram<T>(cluster, rl, 0, 0, rl, nrows, true, &S.inbox[0][0][0], nwr);
    cluster.sync();
    reduce_inbox<T>(&S.inbox[0][0][0], ncta, 1, S.red, nwr);
    const double nb = sqrt(fmax((double)S.red[0].x, 0.0));
    const double tol_abs = a.tol * nb;
    int iters = 0, cycles = 0, conv = 0, stop_next = 0;
    // test probe: a bounded wait on a barrier that nothing completes
    if (flow && a.probe && !ls_warp && !S.fault && !mbar_wait(&S.mb[3], 0u, spin)) S.fault = 1;
    __syncthreads();
    // Least-squares update of step jc by one warp (lane = 0..31): column jc of H
    // (h1 + h2, h_{jc+1,jc}), the previous rotations applied to it, the new
    // rotation, and the stop flags from the residual estimate |g_{jc+1}|.  Reads
    // S.h1 and S.red, which the step after jc overwrites only after its apply.
    auto ls_update = [&](int lane, int jc, T hnv) {
        for (int i = lane; i <= jc; i += 32) st.H[i + LD * jc] = cadd(S.h1[i], S.red[i]);
        if (lane == 0) st.H[(jc + 1) + LD * jc] = mk<T>(hnv, 0);
        __syncwarp();
        if (lane == 0) {
            // distinct arrays: the loads of later rotations need not wait for the
            // stores of earlier ones
            const Z* __restrict__ Hc = st.H + LD * jc;
            Z* __restrict__ Rc = st.Rm + LD * jc;
            const T* __restrict__ rcs = st.rc;
            const Z* __restrict__ rss = st.rs;
            Z p = Hc[0];
#pragma unroll 8
            for (int t = 0; t < jc; ++t) {
                Z q = Hc[t + 1];
                rot_<T>(rcs[t], rss[t], p, q);
                Rc[t] = p;
                p = q;
            }
            T cc;
            Z ss, rr;
            givens_real_<T>(p, hnv, cc, ss, rr);
            Rc[jc] = rr;
            st.rc[jc] = cc;
            st.rs[jc] = ss;
            rot_<T>(cc, ss, st.g[jc], st.g[jc + 1]);
            const Z gn = st.g[jc + 1];
            S.ctl[0] = ((double)(gn.x * gn.x + gn.y * gn.y) <= tol_abs * tol_abs) ? 1 : 0;
            S.ctl[1] = (hnv == T(0)) ? 1 : 0;
        }
        __syncwarp();
    };
    // The same Givens update for a column jc of H that the row warps have already
    // written in full (delayed CGS2), with subdiagonal hnv
    auto ls_col = [&](int lane, int jc, T hnv) {
        if (lane == 0) {
            const Z* __restrict__ Hc = st.H + LD * jc;
            Z* __restrict__ Rc = st.Rm + LD * jc;
            const T* __restrict__ rcs = st.rc;
            const Z* __restrict__ rss = st.rs;
            Z p = Hc[0];
#pragma unroll 8
            for (int t = 0; t < jc; ++t) {
                Z q = Hc[t + 1];
                rot_<T>(rcs[t], rss[t], p, q);
                Rc[t] = p;
                p = q;
            }
            T cc;
            Z ss, rr;
            givens_real_<T>(p, hnv, cc, ss, rr);
            Rc[jc] = rr;
            st.rc[jc] = cc;
            st.rs[jc] = ss;
            rot_<T>(cc, ss, st.g[jc], st.g[jc + 1]);
            const Z gn = st.g[jc + 1];
            S.ctl[0] = ((double)(gn.x * gn.x + gn.y * gn.y) <= tol_abs * tol_abs) ? 1 : 0;
            S.ctl[1] = (hnv == T(0)) ? 1 : 0;
        }
        __syncwarp();
    };
    // delayed CGS2 (a.dc, dataflow push mode only): one exchange per Arnoldi step
    const bool dc = flow && a.lsw && a.dc;
    // w = A v (push mode: v staged in xs) on the CTA's rows, then a CTA barrier
    auto dc_apply = [&](Z* out) {
        for (int e = tid; e < nrows; e += nt) {
            const int ls = e / NDOF, kk = e - ls * NDOF;
            Z acc = mk<T>(0, 0);
            if (a.Ah) {
                const unsigned* Ab = a.Ah + (s0 + ls) * (5L * NDOF * NDOF) + kk;
                if (a.ash) {
                    const unsigned* As = Ash + ls * ASH_SITE_WORDS + kk;
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
#pragma unroll
                        for (int l = 0; l < NDOF; ++l) {
                            const Z av = d < ASH_DIRS ? half_bits<T>(As[(d * NDOF + l) * NDOF])
                                                      : half_entry<T>(Ab + (d * NDOF + l) * NDOF);
                            acc = cfma(av, S.xs[ls][d][l], acc);
                        }
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
#pragma unroll
                        for (int l = 0; l < NDOF; ++l)
                            acc = cfma(half_entry<T>(Ab + (d * NDOF + l) * NDOF), S.xs[ls][d][l], acc);
                    }
                }
            } else {
                const Z* Ab = a.A + (s0 + ls) * (5L * NDOF * NDOF) + kk;
#pragma unroll
                for (int d = 0; d < 5; ++d) {
#pragma unroll
                    for (int l = 0; l < NDOF; ++l) acc = cfma(__ldg(Ab + (d * NDOF + l) * NDOF), S.xs[ls][d][l], acc);
                }
            }
            out[e] = acc;
        }
        __syncthreads();
    };
    // One GMRES(ms) cycle with delayed CGS2 from v_0 (row 0, staged): step j applies
    // A to u_j, the once-orthogonalised next vector, and one exchange gives
    // a = Q_{j-1}^+ u_j, |u_j|^2, Q_{j-1}^+ w and u_j^+ w.  That finishes q_j
    // (the second pass of step j - 1) and column j - 1 of H; A q_j then follows
    // from the Arnoldi relation, A q_j = (w - Q_j H a) / rho, and its first
    // projection gives u_{j+1}.  The least-squares warp updates column j - 1
    // during the rest of step j; its stop flags are read at step j + 1's apply
    // barrier.  The inboxes alternate by step (buffer reuse stays safe as in the
    // two-exchange step).  Returns the number of finished columns.
    auto dcgs2_cycle = [&]() -> int {
        const int lane = tid & 31;
        Z* const ib[2] = {&S.inbox[0][0][0], &S.inbox[1][0][0]};
        const unsigned zb = (unsigned)sizeof(Z);
        const unsigned stage_bytes = (unsigned)(my_sites * 5 * NDOF) * zb;
        // step 0: w = A q_0, h = q_0^+ w, u_1 = w - q_0 h
        {
            Z* const w = Vl + ldv;
            dc_apply(w);
            arm(0, (unsigned)ncta * zb);
            push_gram_flow<T>(Vl, ldv, 1, w, nrows, false, ib[0], &S.mb[0], ncta, rank, nwr);
            if (!ls_warp) flow_wait(0);
            reduce_inbox<T>(ib[0], ncta, 1, S.h1, nwr);
            arm(2, stage_bytes);
            for (int e = tid; e < nrows; e += nt) {
                const Z v = accum_rows<T, true>(w[e], Vl, ldv, e, S.h1, 1);
                w[e] = v;
                push_row_flow<T>(S, e, v, mma);
            }
        }
        for (int j = 1; j < ms; ++j) {
            Z* const u = Vl + (long)j * ldv;
            Z* const wl = Vl + (long)(j + 1) * ldv;
            if (!ls_warp) flow_wait(2);  // u_j staged from every neighbour
            dc_apply(wl);
            if (j >= 2 && (S.ctl[0] | S.ctl[1])) {  // column j - 2 ended the cycle
                conv = S.ctl[0];
                return j - 1;
            }
            const int b = j & 1;
            arm(b, (unsigned)(ncta * (2 * j + 2)) * zb);
            push_gram_flow<T>(Vl, ldv, j, u, nrows, true, ib[b], &S.mb[b], ncta, rank, nwr);
            push_gram_flow<T>(Vl, ldv, j + 1, wl, nrows, false, ib[b] + (j + 1), &S.mb[b], ncta, rank, nwr);
            if (!ls_warp) flow_wait(b);
            reduce_inbox<T>(ib[b], ncta, 2 * j + 2, S.red, nwr);  // a | |u|^2 | Q^+ w | u^+ w
            T aa = 0;
            Z ab = mk<T>(0, 0);
            for (int i = lane; i < j; i += 32) {
                aa += S.red[i].x * S.red[i].x + S.red[i].y * S.red[i].y;
                ab = cfmac(S.red[i], S.red[j + 1 + i], ab);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                aa += __shfl_xor_sync(0xffffffffu, aa, o);
                ab.x += __shfl_xor_sync(0xffffffffu, ab.x, o);
                ab.y += __shfl_xor_sync(0xffffffffu, ab.y, o);
            }
            const T rho = sqrt(fmax((T)S.red[j].x - aa, T(0)));
            const T irho = rho > T(0) ? T(1) / rho : T(0);
            for (int e = tid; e < nrows; e += nt) u[e] = cscale(accum_rows<T, true>(u[e], Vl, ldv, e, S.red, j), irho);
            if (tid < j) st.H[tid + LD * (j - 1)] = cadd(S.h1[tid], S.red[tid]);
            if (tid == j) st.H[j + LD * (j - 1)] = mk<T>(rho, 0);
            __syncthreads();  // q_j and column j - 1 complete
            if (ls_warp) {
                ls_col(lane, j - 1, rho);
            } else {
                if (tid <= j) {
                    Z y = mk<T>(0, 0);
                    for (int l = (tid > 0 ? tid - 1 : 0); l < j; ++l) y = cfma(st.H[tid + LD * l], S.red[l], y);
                    const Z qw = tid < j ? S.red[j + 1 + tid] : cscale(csub(S.red[2 * j + 1], ab), irho);
                    const Z h = cscale(csub(qw, y), irho);
                    S.hnext[tid] = h;
                    S.zc[tid] = cadd(y, cscale(h, rho));
                }
                row_warps_sync(nwr * 32);
                if (tid <= j) S.h1[tid] = S.hnext[tid];
                arm(2, stage_bytes);
                for (int e = tid; e < nrows; e += nwr * 32) {  // row warps only
                    const Z v = cscale(accum_rows<T, true>(wl[e], Vl, ldv, e, S.zc, j + 1), irho);
                    wl[e] = v;
                    push_row_flow<T>(S, e, v, mma);
                }
            }
            ++iters;
        }
        // u_ms is staged, and no apply reads it
        if (!ls_warp) flow_wait(2);
        __syncthreads();  // the update of column ms - 2 is complete
        if (ms >= 2 && (S.ctl[0] | S.ctl[1])) {
            conv = S.ctl[0];
            return ms - 1;
        }
        // the last second pass: q_ms and column ms - 1
        const int b = ms & 1;
        Z* const u = Vl + (long)ms * ldv;
        arm(b, (unsigned)(ncta * (ms + 1)) * zb);
        push_gram_flow<T>(Vl, ldv, ms, u, nrows, true, ib[b], &S.mb[b], ncta, rank, nwr);
        if (!ls_warp) flow_wait(b);
        reduce_inbox<T>(ib[b], ncta, ms + 1, S.red, nwr);
        T aa = 0;
        for (int i = lane; i < ms; i += 32) aa += S.red[i].x * S.red[i].x + S.red[i].y * S.red[i].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) aa += __shfl_xor_sync(0xffffffffu, aa, o);
        const T rho = sqrt(fmax((T)S.red[ms].x - aa, T(0)));
        const T irho = rho > T(0) ? T(1) / rho : T(0);
        for (int e = tid; e < nrows; e += nt) u[e] = cscale(accum_rows<T, true>(u[e], Vl, ldv, e, S.red, ms), irho);
        if (tid < ms) st.H[tid + LD * (ms - 1)] = cadd(S.h1[tid], S.red[tid]);
        if (tid == ms) st.H[ms + LD * (ms - 1)] = mk<T>(rho, 0);
        __syncthreads();
        if (ls_warp) ls_col(lane, ms - 1, rho);
        __syncthreads();
        ++iters;
        conv = S.ctl[0];
        return ms;
    };
    while (true) {
        // ---- projection onto the deflation space: d = argmin ||W^+ r - H_k d|| ----
        if (tid == 0) S.fpub[cycles & 1] = S.fault;
        push_gram<T>(cluster, Wl, ldw, k + 1, rl, nrows, false, &S.inbox[1][0][0], nwr);
        cluster.sync();
        // Leave together: a fault anywhere in the cluster (each CTA published its
        // flag before this barrier, in the slot of this cycle's parity, which no
        // CTA rewrites before the next barrier), or the previous cycle's stop,
        // which every CTA took from identical data when none faulted.
        if (flow) {
            int anyf = 0;
            for (int q = 0; q < ncta; ++q) anyf |= *cluster.map_shared_rank(&S.fpub[cycles & 1], q);
            if (anyf) break;
        }
        if (stop_next) break;
        reduce_inbox<T>(&S.inbox[1][0][0], ncta, k + 1, S.red, nwr);
        for (int i = tid; i <= k; i += nt) {
            Z pdv = mk<T>(0, 0), puv = mk<T>(0, 0);
            for (int l = 0; l <= k; ++l) {
                const Z gl = S.red[l];
                if (i < k) pdv = cfma(Mp[i + k * l], gl, pdv);
                puv = cfma(Np[i + (k + 1) * l], gl, puv);
            }
            if (i < k) st.pd[i] = pdv;
            st.pu[i] = puv;
        }
        __syncthreads();
        for (int e = tid; e < nrows; e += nt) {
            xl[e] = accum_rows<T, false>(xl[e], Wl, ldw, e, st.pd, k);
            rl[e] = accum_rows<T, true>(rl[e], Wl, ldw, e, st.pu, k + 1);
        }
        __syncthreads();
        push_gram<T>(cluster, rl, 0, 0, rl, nrows, true, &S.inbox[0][0][0], nwr);
        cluster.sync();
        reduce_inbox<T>(&S.inbox[0][0][0], ncta, 1, S.red, nwr);
        // beta = ||r|| (FP64 square root and division: thread 0 alone, as the
        // FP64 units are few), the stop test, and the start of the cycle
        if (tid == 0) {
            const double beta = sqrt(fmax((double)S.red[0].x, 0.0));
            const int done = (beta <= tol_abs || beta == 0.0) ? 1 : 0;
            S.ctl[2] = done;
            if (!done) {
                for (int i = 0; i <= ms; ++i) {
                    st.c[i] = mk<T>(i == 0 ? (T)beta : T(0), 0);
                    st.g[i] = st.c[i];
                }
                S.scal[0] = (T)(1.0 / beta);
                S.ctl[0] = S.ctl[1] = 0;
            }
        }
        // ---- one GMRES(ms) cycle from r ----
        // (shared memory is not zero-initialised: H must be zero below its subdiagonal)
        for (int e = tid; e < LD * MSMAX; e += nt) {
            st.H[e] = mk<T>(0, 0);
            st.Rm[e] = mk<T>(0, 0);
        }
        __syncthreads();
        if (S.ctl[2]) {
            conv = 1;
            break;
        }
        {
            const T sc = S.scal[0];
            for (int e = tid; e < nrows; e += nt) {
                const Z v = cscale(rl[e], sc);
                Vl[e] = v;
                if (push)
                    push_row<T>(S, rank, e, v, mma);
                else if (a.vs)
                    a.V[r0 + e] = v;
            }
        }
        cluster.sync();  // v_0 complete in every CTA
        int j = 0, stop = 0;
        if (dc) {
            j = dcgs2_cycle();
        } else {
        for (; j < ms && !stop; ++j) {
            const Z* vj = a.V + (long)j * n;
            Z* wl = Vl + (long)(j + 1) * ldv;
            // w = A v_j on the CTA's rows (column-major 24x24 blocks), MAX_SPC sites at a
            // time: stage the five neighbour rows of each site (other CTAs' rows: through L2)
            CP_STAMP(6);
            if (flow && j > 0 && !ls_warp) flow_wait(2);  // v_j staged from every neighbour
            CP_STAMP(0);
            for (int c0 = 0; c0 < my_sites; c0 += MAX_SPC) {
                const int cs = min(MAX_SPC, my_sites - c0);
                if (!push) {
                    for (int e = tid; e < cs * 5 * NDOF; e += nt) {
                        const int ls = e / (5 * NDOF), rem = e - ls * 5 * NDOF, d = rem / NDOF, l = rem - d * NDOF;
                        const long nbs = table ? (long)S.nbt[c0 + ls][d] : nbr_site(s0 + c0 + ls, d, a.Nx, a.Nt);
                        S.xs[ls][d][l] = __ldcg(vj + nbs * NDOF + l);
                    }
                    __syncthreads();
                }
                if (mma) {  // push mode: c0 == 0, cs == my_sites
                    if constexpr (std::is_same<T, float>::value) {
                        // one site per row warp at a time; its streamed fragments are
                        // loaded first and arrive during the shared-memory directions
                        const int lane = tid & 31;
                        if ((tid >> 5) < nwr)
                            for (int ls = tid >> 5; ls < cs; ls += nwr) {
                                unsigned f[TC_SW];
                                tc_load_stream(a.Ah + (s0 + ls) * (5L * NDOF * NDOF), f, lane);
                                TcAcc c;
                                tc_zero(c);
                                tc_shared_dirs(c, Ash + ls * ASH_SITE_WORDS, S.xs[ls], lane);
                                tc_stream_dirs(c, f, S.xs[ls], lane);
                                tc_store(c, wl + (long)ls * NDOF, lane);
                            }
                    }
                } else if (a.Ah) {  // FP16 operator copy: half the bytes of the stream, FP32 arithmetic
                    for (int e = tid; e < cs * NDOF; e += nt) {
                        const int ls = e / NDOF, kk = e - ls * NDOF;
                        const unsigned* Ab = a.Ah + (s0 + c0 + ls) * (5L * NDOF * NDOF) + kk;
                        Z acc = mk<T>(0, 0);
                        if (a.ash) {  // push mode: c0 == 0
                            const unsigned* As = Ash + ls * ASH_SITE_WORDS + kk;
#pragma unroll
                            for (int d = 0; d < 5; ++d) {
#pragma unroll
                                for (int l = 0; l < NDOF; ++l) {
                                    const Z av = d < ASH_DIRS ? half_bits<T>(As[(d * NDOF + l) * NDOF])
                                                              : half_entry<T>(Ab + (d * NDOF + l) * NDOF);
                                    acc = cfma(av, S.xs[ls][d][l], acc);
                                }
                            }
                        } else {
#pragma unroll
                            for (int d = 0; d < 5; ++d) {
#pragma unroll
                                for (int l = 0; l < NDOF; ++l)
                                    acc = cfma(half_entry<T>(Ab + (d * NDOF + l) * NDOF), S.xs[ls][d][l], acc);
                            }
                        }
                        wl[(long)c0 * NDOF + e] = acc;
                    }
                } else {
                    for (int e = tid; e < cs * NDOF; e += nt) {
                        const int ls = e / NDOF, kk = e - ls * NDOF;
                        const Z* Ab = a.A + (s0 + c0 + ls) * (5L * NDOF * NDOF) + kk;
                        Z acc = mk<T>(0, 0);
#pragma unroll
                        for (int d = 0; d < 5; ++d) {
#pragma unroll
                            for (int l = 0; l < NDOF; ++l)
                                acc = cfma(__ldg(Ab + (d * NDOF + l) * NDOF), S.xs[ls][d][l], acc);
                        }
                        wl[(long)c0 * NDOF + e] = acc;
                    }
                }
                __syncthreads();
            }
            CP_STAMP(1);
            if (a.lsw && j > 0) {  // step j - 1's update is complete (apply barrier)
                conv = S.ctl[0];
                if (S.ctl[0] | S.ctl[1]) break;  // step j is discarded: j columns
            }
            if (flow) {
                arm(1, (unsigned)(ncta * (j + 1) * sizeof(Z)));
                push_gram_flow<T>(Vl, ldv, j + 1, wl, nrows, false, &S.inbox[1][0][0], &S.mb[1], ncta, rank, nwr);
                if (!ls_warp) flow_wait(1);
            } else {
                push_gram<T>(cluster, Vl, ldv, j + 1, wl, nrows, false, &S.inbox[1][0][0], nwr);
                cluster.sync();
            }
            CP_STAMP(2);
            reduce_inbox<T>(&S.inbox[1][0][0], ncta, j + 1, S.h1, nwr);
            for (int e = tid; e < nrows; e += nt) wl[e] = accum_rows<T, true>(wl[e], Vl, ldv, e, S.h1, j + 1);
            __syncthreads();
            CP_STAMP(3);
            if (flow) {
                arm(0, (unsigned)(ncta * (j + 2) * sizeof(Z)));
                push_gram_flow<T>(Vl, ldv, j + 1, wl, nrows, true, &S.inbox[0][0][0], &S.mb[0], ncta, rank, nwr);
                if (!ls_warp) flow_wait(0);
            } else {
                push_gram<T>(cluster, Vl, ldv, j + 1, wl, nrows, true, &S.inbox[0][0][0], nwr);
                cluster.sync();
            }
            CP_STAMP(4);
            reduce_inbox<T>(&S.inbox[0][0][0], ncta, j + 2, S.red, nwr);
            // h_{j+1,j} = ||w - V h2|| = sqrt(n2 - |h2|^2) (V orthonormal), computed
            // identically by every thread; then v_{j+1} = (w - V h2) / h_{j+1,j}
            T h2n = 0;  // warp butterfly: the same value in every lane and warp
            for (int i = tid & 31; i <= j; i += 32) h2n += S.red[i].x * S.red[i].x + S.red[i].y * S.red[i].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) h2n += __shfl_xor_sync(0xffffffffu, h2n, o);
            const T hn = sqrt(fmax((T)S.red[j + 1].x - h2n, T(0)));
            {
                const T sc = hn > T(0) ? T(1) / hn : T(0);
                Z* wg = a.V + (long)(j + 1) * n + r0;
                if (flow) arm(2, (unsigned)(my_sites * 5 * NDOF * sizeof(Z)));
                for (int e = tid; e < nrows; e += nt) {
                    const Z v = cscale(accum_rows<T, true>(wl[e], Vl, ldv, e, S.red, j + 1), sc);
                    wl[e] = v;
                    if (flow)
                        push_row_flow<T>(S, e, v, mma);
                    else if (push)
                        push_row<T>(S, rank, e, v, mma);
                    else if (a.vs)
                        wg[e] = v;
                }
            }
            CP_STAMP(5);
#ifdef CP_PHASE_CLOCKS
            ++clk_steps;
#endif
            if (flow) {
                // no barrier: the next apply waits for its staging slots instead; the
                // least-squares warp updates step j meanwhile
                if (ls_warp) ls_update(tid & 31, j, hn);
                ++iters;
                continue;
            }
            __syncwarp();
            cluster_arrive();  // v_{j+1} complete in this CTA
            if (a.lsw) {
                cluster_wait();  // v_{j+1} complete in every CTA
                // the least-squares warp updates step j while the row warps go on to
                // step j + 1; its stop flags are read after that step's apply
                if (ls_warp) ls_update(tid & 31, j, hn);
                ++iters;
            } else {
                // warp 0 updates the least squares between arrive and wait
                if (tid < 32) ls_update(tid, j, hn);
                cluster_wait();  // v_{j+1} complete in every CTA
                __syncthreads();
                ++iters;
                conv = S.ctl[0];
                stop = S.ctl[0] | S.ctl[1];
            }
        }
        if (a.lsw && j == ms) {  // the last step's update, when no stop came before
            if (flow && !ls_warp) flow_wait(2);  // the staging of v_ms, which no apply reads
            __syncthreads();
            conv = S.ctl[0];
        }
        }
        // ---- finish the cycle: d = R^{-1} g, rho = c - H d, x += V d, r = V rho ----
        const int jj = j;
        if (tid < 32) back_subst_warp<T>(st.Rm, st.g, st.d, jj, tid);
        __syncthreads();
        for (int i = tid; i <= jj; i += nt) {
            Z acc = st.c[i];
            for (int l = 0; l < jj; ++l) acc = cfms_<T>(st.H[i + LD * l], st.d[l], acc);
            st.rho[i] = acc;
        }
        __syncthreads();
        for (int e = tid; e < nrows; e += nt) {
            xl[e] = accum_rows<T, false>(xl[e], Vl, ldv, e, st.d, jj);
            rl[e] = accum_rows<T, false>(mk<T>(0, 0), Vl, ldv, e, st.rho, jj + 1);
        }
        ++cycles;
        __syncthreads();
        stop_next = (conv || cycles >= a.max_cycles) ? 1 : 0;  // taken after the next cluster barrier
    }
    __syncthreads();
    if (flow && tid == 0 && S.fault) atomicAdd(reinterpret_cast<unsigned long long*>(&a.out->timeouts), 1ULL);
    if (rank == 0 && tid == 0) {
        a.out->iters += iters;
        a.out->cycles += cycles;
        a.out->solves += 1;
        a.out->unconverged += conv ? 0 : 1;
        a.out->ctas = ncta;
        a.out->spc = a.spc;
        a.out->flow = flow ? 1 : 0;
        a.out->dc = dc ? 1 : 0;
        a.out->ash = a.ash;
        a.out->half = a.Ah ? 1 : 0;
        a.out->paired = 0;
        a.out->mma = mma ? 1 : 0;
    }
#ifdef CP_PHASE_CLOCKS
    if (clk && clk_steps > 0)
        printf("coarse_proj phases (cycles/step over %d steps, mma %d): staging wait %lld, apply %lld, gram1+wait %lld, "
               "reduce+update %lld, gram2+wait %lld, reduce+v+push %lld, other %lld\n",
               clk_steps, mma ? 1 : 0, acc_t[0] / clk_steps, acc_t[1] / clk_steps, acc_t[2] / clk_steps,
               acc_t[3] / clk_steps, acc_t[4] / clk_steps, acc_t[5] / clk_steps, acc_t[6] / clk_steps);
#endif
    cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------------------
// Two right-hand sides of one coarsest operator in lockstep (FP32, push mode).
// Both solves run the same GMRES-Proj algorithm as k_coarse_proj, step for
// step and with the same arithmetic per right-hand side (so each result equals
// the single kernel's); they share the operator stream of the apply (each
// block entry is loaded once and used for both vectors) and the cluster
// barriers.  A solve that has stopped its cycle, or converged, idles through
// the other's steps.

template <typename T>
struct PairSmem {
    C2<T> inbox[2][2][MAX_CLUSTER][PSTR];  // [phase][rhs]: partial sums pushed by every CTA
    C2<T> red[2][PSTR];
    C2<T> h1[2][MSMAX + 1];
    C2<T> xs[2][MAX_SPC][5][NDOF];
    int pusht[MAX_SPC][5];
    Small<T> st[2];
    T scal[2][8];
    int ctl[2][8];
    unsigned long long mb[3];  // dataflow mode, as in ClusterSmem
    int fault;
    int fpub[2];               // fault as published at a cycle's first cluster barrier, as in ClusterSmem
};

// push_gram for the two right-hand sides at once: warp task i forms product i
// (basis vector i, or the norm when i == nd) of both right-hand sides, their
// loads and shuffles interleaved; act[b] == 0 skips rhs b.  Per right-hand side
// the summation order is push_gram's.
template <typename T>
__device__ void push_gram2(const C2<T>* const X[2], long ldx, int nd, const C2<T>* const y[2], int nrows, bool norm,
                           C2<T>* const inbox[2], const int act[2], int nr, int me, int nw,
                           unsigned long long* bar = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = nd + (norm ? 1 : 0);
    const bool on0 = act[0] != 0, on1 = act[1] != 0;
    if (!on0 && !on1) return;
    // an idle right-hand side reads the active one's vectors (never stored)
    const int b0 = on0 ? 0 : 1, b1 = on1 ? 1 : 0;
    const C2<T>* y0 = y[b0];
    const C2<T>* y1 = y[b1];
    for (int i = warp; i < per; i += nw) {
        C2<T> p4[4], q4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p4[u] = q4[u] = mk<T>(0, 0);
        const C2<T>* x0 = (i < nd) ? X[b0] + (long)i * ldx : y0;
        const C2<T>* x1 = (i < nd) ? X[b1] + (long)i * ldx : y1;
        int e = lane;
        for (; e + 96 < nrows; e += 128) {
            C2<T> xa[4], ya[4], xb[4], yb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = x0[e + 32 * u];
                ya[u] = y0[e + 32 * u];
                xb[u] = x1[e + 32 * u];
                yb[u] = y1[e + 32 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p4[u] = cfmac(xa[u], ya[u], p4[u]);
                q4[u] = cfmac(xb[u], yb[u], q4[u]);
            }
        }
        for (; e < nrows; e += 32) {
            p4[0] = cfmac(x0[e], y0[e], p4[0]);
            q4[0] = cfmac(x1[e], y1[e], q4[0]);
        }
        C2<T> p = cadd(cadd(p4[0], p4[1]), cadd(p4[2], p4[3]));
        C2<T> q = cadd(cadd(q4[0], q4[1]), cadd(q4[2], q4[3]));
        if (i >= nd) p.y = q.y = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p.x += __shfl_xor_sync(0xffffffffu, p.x, o);
            p.y += __shfl_xor_sync(0xffffffffu, p.y, o);
            q.x += __shfl_xor_sync(0xffffffffu, q.x, o);
            q.y += __shfl_xor_sync(0xffffffffu, q.y, o);
        }
        if (lane < nr) {
            if (bar) {  // dataflow mode: st.async counted on the receiver's barrier
                const unsigned br = cluster_addr(smem_addr(bar), lane);
                if (on0) st_async(cluster_addr(smem_addr(inbox[0] + me * PSTR + i), lane), p, br);
                if (on1) st_async(cluster_addr(smem_addr(inbox[1] + me * PSTR + i), lane), q, br);
            } else {
                if (on0) st_rank<T>(inbox[0] + me * PSTR + i, lane, me, p);
                if (on1) st_rank<T>(inbox[1] + me * PSTR + i, lane, me, q);
            }
        }
    }
}

// reduce_inbox for the two right-hand sides (warp task i sums entry i of both,
// same tree as the single kernel), then a block barrier
template <typename T>
__device__ void reduce_inbox2(C2<T>* const inbox[2], int nr, int n, C2<T>* const red[2], const int act[2], int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool on0 = act[0] != 0, on1 = act[1] != 0;
    if (on0 || on1)
        for (int i = warp; i < n; i += nw) {
            C2<T> p = mk<T>(0, 0), q = mk<T>(0, 0);
            if (lane < nr) {
                if (on0) p = inbox[0][lane * PSTR + i];
                if (on1) q = inbox[1][lane * PSTR + i];
            }
#pragma unroll
            for (int o = MAX_CLUSTER / 2; o > 0; o >>= 1) {
                p.x += __shfl_xor_sync(0xffffffffu, p.x, o);
                p.y += __shfl_xor_sync(0xffffffffu, p.y, o);
                q.x += __shfl_xor_sync(0xffffffffu, q.x, o);
                q.y += __shfl_xor_sync(0xffffffffu, q.y, o);
            }
            if (lane == 0) {
                if (on0) red[0][i] = p;
                if (on1) red[1][i] = q;
            }
        }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void push_row2(PairSmem<T>& S, int me, int b, int e, C2<T> v, bool flow = false) {
    const int ls = e / NDOF, kk = e - ls * NDOF;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int code = S.pusht[ls][q], owner = code >> 16;
        C2<T>* dst = &S.xs[b][(code >> 3) & 0x1fff][code & 7][kk];
        if (flow)
            st_async(cluster_addr(smem_addr(dst), owner), v, cluster_addr(smem_addr(&S.mb[2]), owner));
        else
            st_rank<T>(dst, owner, me, v);
    }
}

template <typename T>
__global__ void __maxnreg__(128) k_coarse_proj_pair(CoopArgs<T> a0, CoopArgs<T> a1) {
    using Z = C2<T>;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PairSmem<T>& S = *reinterpret_cast<PairSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int rank = (int)cluster.block_rank(), ncta = (int)cluster.num_blocks();
    const long nsite = (long)a0.Nx * a0.Nt;
    const long n = nsite * NDOF;
    const long s0 = (long)rank * a0.spc;
    const long s1 = min(nsite, s0 + a0.spc);
    const int my_sites = (int)max(0L, s1 - s0);
    const long r0 = s0 * NDOF;
    const int nrows = my_sites * NDOF;
    const int k = a0.k, ms = a0.ms;
    const int LD = MSMAX + 1;
    const int rows_cap = a0.spc * NDOF;
    const long ldv = rows_cap;
    Z* Vb[2];
    Vb[0] = reinterpret_cast<Z*>(smem_raw + sizeof(PairSmem<T>));
    Vb[1] = Vb[0] + (long)(ms + 1) * rows_cap;
    const Z* Wl = a0.W + r0;
    const long ldw = n;
    Z* xl[2] = {a0.x + r0, a1.x + r0};
    Z* rl[2] = {a0.r + r0, a1.r + r0};
    const Z* fl[2] = {a0.f + r0, a1.f + r0};
    const double tol_rel[2] = {a0.tol, a1.tol};
    for (int e = tid; e < my_sites * 5; e += nt) {  // push table, as in k_coarse_proj
        const int ls = e / 5, q = e - ls * 5;
        const int from[5] = {0, 2, 1, 4, 3};
        const long w = nbr_site(s0 + ls, from[q], a0.Nx, a0.Nt);
        const int owner = (int)(w / a0.spc);
        S.pusht[ls][q] = (owner << 16) | ((int)(w - (long)owner * a0.spc) << 3) | q;
    }
    // dataflow mode for the exchanges of each Arnoldi step, as in k_coarse_proj
    // (one barrier a phase for both right-hand sides: bytes of the active ones)
    const bool flow = a0.flow != 0;
    const long spin = a0.spin > 0 ? a0.spin : FLOW_SPIN;
    unsigned fph[3] = {0u, 0u, 0u};
    // a wait that gives up marks the CTA faulted, as in k_coarse_proj
    auto flow_wait = [&](int b) {
        if (!S.fault && !mbar_wait(&S.mb[b], fph[b], spin)) S.fault = 1;
        fph[b] ^= 1u;
    };
    auto arm = [&](int b, unsigned bytes) {
        if (tid == 0 && !S.fault) mbar_arm(&S.mb[b], bytes);
    };
    if (tid == 0) {
        if (flow) {
            for (int b = 0; b < 3; ++b) mbar_init(&S.mb[b], 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        S.fault = 0;
        S.fpub[0] = S.fpub[1] = 0;
    }
    // projection matrices M, N (shared deflation space), as in k_coarse_proj
    Z* Mp = Vb[1] + (long)(ms + 1) * rows_cap;
    Z* Np = Mp + k * (k + 1);
    if (tid < 32) {
        const KState* P = a0.pls;
        for (int l = tid; l <= k; l += 32) {
            Z g[KLD], dd[KMAX];
            for (int i = 0; i <= k; ++i) g[i] = mk<T>(i == l ? T(1) : T(0), 0);
            for (int t = 0; t < P->nrot; ++t)
                rot_<T>((T)P->rc[t], from_d2<T>(P->rs[t]), g[P->ra[t]], g[P->rb[t]]);
            for (int i = k - 1; i >= 0; --i) {
                Z acc = g[i];
                for (int m = i + 1; m < k; ++m) acc = cfms_<T>(from_d2<T>(P->R[i + KLD * m]), dd[m], acc);
                dd[i] = cdiv_<T>(acc, from_d2<T>(P->R[i + KLD * i]));
            }
            for (int i = 0; i < k; ++i) Mp[i + k * l] = dd[i];
            for (int i = 0; i <= k; ++i) {
                Z acc = mk<T>(0, 0);
                for (int m = 0; m < k; ++m) acc = cfma(from_d2<T>(P->H[i + KLD * m]), dd[m], acc);
                Np[i + (k + 1) * l] = acc;
            }
        }
    }
    for (int e = tid; e < 2 * nrows; e += nt) {  // x = 0, r = f
        const int b = e / nrows, rr = e - b * nrows;
        xl[b][rr] = mk<T>(0, 0);
        rl[b][rr] = fl[b][rr];
    }
    __syncthreads();
    int act[2] = {1, 1}, conv[2] = {0, 0}, iters[2] = {0, 0};
    const int all2[2] = {1, 1};
    C2<T>* const in0[2] = {&S.inbox[0][0][0][0], &S.inbox[0][1][0][0]};
    C2<T>* const in1[2] = {&S.inbox[1][0][0][0], &S.inbox[1][1][0][0]};
    C2<T>* const redp[2] = {S.red[0], S.red[1]};
    C2<T>* const h1p[2] = {S.h1[0], S.h1[1]};
    const Z* const rlc[2] = {rl[0], rl[1]};
    push_gram2<T>(rlc, 0, 0, rlc, nrows, true, in0, all2, ncta, rank, nw);
    cluster.sync();
    reduce_inbox2<T>(in0, ncta, 1, redp, all2, nw);
    double tol_abs[2];
    for (int b = 0; b < 2; ++b) tol_abs[b] = tol_rel[b] * sqrt(fmax((double)S.red[b][0].x, 0.0));
    int cycles = 0;
    while (true) {
        // ---- projection onto the shared deflation space, per right-hand side ----
        const Z* const Wb[2] = {Wl, Wl};
        if (tid == 0) S.fpub[cycles & 1] = S.fault;
        push_gram2<T>(Wb, ldw, k + 1, rlc, nrows, false, in1, act, ncta, rank, nw);
        cluster.sync();
        // leave together on a fault anywhere in the cluster, as in k_coarse_proj;
        // the stops of the previous cycle take effect here too
        if (flow) {
            int anyf = 0;
            for (int q = 0; q < ncta; ++q) anyf |= *cluster.map_shared_rank(&S.fpub[cycles & 1], q);
            if (anyf) break;
        }
        for (int b = 0; b < 2; ++b)
            if (act[b] && (conv[b] || cycles >= a0.max_cycles)) act[b] = 0;
        if (!act[0] && !act[1]) break;
        reduce_inbox2<T>(in1, ncta, k + 1, redp, act, nw);
        for (int t = tid; t < 2 * (k + 1); t += nt) {
            const int b = t / (k + 1), i = t - b * (k + 1);
            if (!act[b]) continue;
            Z pdv = mk<T>(0, 0), puv = mk<T>(0, 0);
            for (int l = 0; l <= k; ++l) {
                const Z gl = S.red[b][l];
                if (i < k) pdv = cfma(Mp[i + k * l], gl, pdv);
                puv = cfma(Np[i + (k + 1) * l], gl, puv);
            }
            if (i < k) S.st[b].pd[i] = pdv;
            S.st[b].pu[i] = puv;
        }
        __syncthreads();
        for (int e = tid; e < 2 * nrows; e += nt) {
            const int b = e / nrows, rr = e - b * nrows;
            if (!act[b]) continue;
            xl[b][rr] = accum_rows<T, false>(xl[b][rr], Wl, ldw, rr, S.st[b].pd, k);
            rl[b][rr] = accum_rows<T, true>(rl[b][rr], Wl, ldw, rr, S.st[b].pu, k + 1);
        }
        __syncthreads();
        push_gram2<T>(rlc, 0, 0, rlc, nrows, true, in0, act, ncta, rank, nw);
        cluster.sync();
        reduce_inbox2<T>(in0, ncta, 1, redp, act, nw);
        // beta_b = ||r_b||, the stop tests and the starts of the cycles, by thread 0
        // (FP64 square root and division), as in k_coarse_proj
        if (tid == 0)
            for (int b = 0; b < 2; ++b) {
                S.ctl[b][2] = 1;
                if (!act[b]) continue;
                const double beta = sqrt(fmax((double)S.red[b][0].x, 0.0));
                if (beta <= tol_abs[b] || beta == 0.0) continue;
                S.ctl[b][2] = 0;
                for (int i = 0; i <= ms; ++i) {
                    S.st[b].c[i] = mk<T>(i == 0 ? (T)beta : T(0), 0);
                    S.st[b].g[i] = S.st[b].c[i];
                }
                S.scal[b][0] = (T)(1.0 / beta);
            }
        // ---- one GMRES(ms) cycle from r for each active right-hand side ----
        for (int e = tid; e < 2 * LD * MSMAX; e += nt) {
            const int b = e / (LD * MSMAX), q = e - b * (LD * MSMAX);
            S.st[b].H[q] = mk<T>(0, 0);
            S.st[b].Rm[q] = mk<T>(0, 0);
        }
        __syncthreads();
        for (int b = 0; b < 2; ++b)
            if (act[b] && S.ctl[b][2]) {
                conv[b] = 1;
                act[b] = 0;
            }
        if (!act[0] && !act[1]) break;
        for (int e = tid; e < 2 * nrows; e += nt) {
            const int b = e / nrows, rr = e - b * nrows;
            if (!act[b]) continue;
            const Z v = cscale(rl[b][rr], S.scal[b][0]);
            Vb[b][rr] = v;
            push_row2<T>(S, rank, b, rr, v);
        }
        cluster.sync();  // v_0 complete in every CTA
        int cact[2] = {act[0], act[1]}, jj[2] = {ms, ms};
        for (int j = 0; j < ms && (cact[0] || cact[1]); ++j) {
            Z* wl[2] = {Vb[0] + (long)(j + 1) * ldv, Vb[1] + (long)(j + 1) * ldv};
            const int nact = cact[0] + cact[1];
            if (flow && j > 0) flow_wait(2);  // v_j of both staged from every neighbour
            // w_b = A v_b: each block entry loaded once for both vectors
            for (int e = tid; e < nrows; e += nt) {
                const int ls = e / NDOF, kk = e - ls * NDOF;
                Z acc0 = mk<T>(0, 0), acc1 = mk<T>(0, 0);
                if (a0.Ah) {  // FP16 operator copy, as in k_coarse_proj
                    const unsigned* Ab = a0.Ah + (s0 + ls) * (5L * NDOF * NDOF) + kk;
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
#pragma unroll
                        for (int l = 0; l < NDOF; ++l) {
                            const Z av = half_entry<T>(Ab + (d * NDOF + l) * NDOF);
                            acc0 = cfma(av, S.xs[0][ls][d][l], acc0);
                            acc1 = cfma(av, S.xs[1][ls][d][l], acc1);
                        }
                    }
                } else {
                    const Z* Ab = a0.A + (s0 + ls) * (5L * NDOF * NDOF) + kk;
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
#pragma unroll
                        for (int l = 0; l < NDOF; ++l) {
                            const Z av = __ldg(Ab + (d * NDOF + l) * NDOF);
                            acc0 = cfma(av, S.xs[0][ls][d][l], acc0);
                            acc1 = cfma(av, S.xs[1][ls][d][l], acc1);
                        }
                    }
                }
                if (cact[0]) wl[0][e] = acc0;
                if (cact[1]) wl[1][e] = acc1;
            }
            __syncthreads();
            const Z* const Vc[2] = {Vb[0], Vb[1]};
            const Z* const wc[2] = {wl[0], wl[1]};
            if (flow) {
                arm(1, (unsigned)(nact * ncta * (j + 1) * sizeof(Z)));
                push_gram2<T>(Vc, ldv, j + 1, wc, nrows, false, in1, cact, ncta, rank, nw, &S.mb[1]);
                flow_wait(1);
            } else {
                push_gram2<T>(Vc, ldv, j + 1, wc, nrows, false, in1, cact, ncta, rank, nw);
                cluster.sync();
            }
            reduce_inbox2<T>(in1, ncta, j + 1, h1p, cact, nw);
            if (cact[0] && cact[1]) {
                for (int rr = tid; rr < nrows; rr += nt) {
                    Z w0 = wl[0][rr], w1 = wl[1][rr];
                    accum_rows2<T, true>(w0, w1, Vb[0], Vb[1], ldv, rr, S.h1[0], S.h1[1], j + 1);
                    wl[0][rr] = w0;
                    wl[1][rr] = w1;
                }
            } else {
                const int b = cact[0] ? 0 : 1;
                for (int rr = tid; rr < nrows; rr += nt)
                    wl[b][rr] = accum_rows<T, true>(wl[b][rr], Vb[b], ldv, rr, S.h1[b], j + 1);
            }
            __syncthreads();
            if (flow) {
                arm(0, (unsigned)(nact * ncta * (j + 2) * sizeof(Z)));
                push_gram2<T>(Vc, ldv, j + 1, wc, nrows, true, in0, cact, ncta, rank, nw, &S.mb[0]);
                flow_wait(0);
            } else {
                push_gram2<T>(Vc, ldv, j + 1, wc, nrows, true, in0, cact, ncta, rank, nw);
                cluster.sync();
            }
            reduce_inbox2<T>(in0, ncta, j + 2, redp, cact, nw);
            T hn[2];
            {  // warp butterfly per right-hand side, as in k_coarse_proj (both at once)
                T h2[2] = {0, 0};
                for (int i = lane; i <= j; i += 32)
#pragma unroll
                    for (int b = 0; b < 2; ++b) h2[b] += S.red[b][i].x * S.red[b][i].x + S.red[b][i].y * S.red[b][i].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int b = 0; b < 2; ++b) h2[b] += __shfl_xor_sync(0xffffffffu, h2[b], o);
#pragma unroll
                for (int b = 0; b < 2; ++b) hn[b] = sqrt(fmax((T)S.red[b][j + 1].x - h2[b], T(0)));
            }
            const T sc[2] = {hn[0] > T(0) ? T(1) / hn[0] : T(0), hn[1] > T(0) ? T(1) / hn[1] : T(0)};
            if (flow) arm(2, (unsigned)(nact * my_sites * 5 * NDOF * sizeof(Z)));
            if (cact[0] && cact[1]) {
                for (int rr = tid; rr < nrows; rr += nt) {
                    Z w0 = wl[0][rr], w1 = wl[1][rr];
                    accum_rows2<T, true>(w0, w1, Vb[0], Vb[1], ldv, rr, S.red[0], S.red[1], j + 1);
                    w0 = cscale(w0, sc[0]);
                    w1 = cscale(w1, sc[1]);
                    wl[0][rr] = w0;
                    wl[1][rr] = w1;
                    push_row2<T>(S, rank, 0, rr, w0, flow);
                    push_row2<T>(S, rank, 1, rr, w1, flow);
                }
            } else {
                const int b = cact[0] ? 0 : 1;
                for (int rr = tid; rr < nrows; rr += nt) {
                    const Z v = cscale(accum_rows<T, true>(wl[b][rr], Vb[b], ldv, rr, S.red[b], j + 1), sc[b]);
                    wl[b][rr] = v;
                    push_row2<T>(S, rank, b, rr, v, flow);
                }
            }
            __syncwarp();
            if (!flow) cluster_arrive();  // dataflow mode: the next apply waits for its slots instead
            // warp b updates the least squares of right-hand side b
            if (warp < 2 && cact[warp]) {
                const int b = warp;
                Small<T>& st = S.st[b];
                for (int i = lane; i <= j; i += 32) st.H[i + LD * j] = cadd(S.h1[b][i], S.red[b][i]);
                if (lane == 0) st.H[(j + 1) + LD * j] = mk<T>(hn[b], 0);
                __syncwarp();
                if (lane == 0) {
                    const Z* __restrict__ Hc = st.H + LD * j;
                    Z* __restrict__ Rc = st.Rm + LD * j;
                    const T* __restrict__ rcs = st.rc;
                    const Z* __restrict__ rss = st.rs;
                    Z p = Hc[0];
#pragma unroll 8
                    for (int t = 0; t < j; ++t) {
                        Z q = Hc[t + 1];
                        rot_<T>(rcs[t], rss[t], p, q);
                        Rc[t] = p;
                        p = q;
                    }
                    T cc;
                    Z ss, rr2;
                    givens_real_<T>(p, hn[b], cc, ss, rr2);
                    Rc[j] = rr2;
                    st.rc[j] = cc;
                    st.rs[j] = ss;
                    rot_<T>(cc, ss, st.g[j], st.g[j + 1]);
                    const Z gn = st.g[j + 1];
                    S.ctl[b][0] = ((double)(gn.x * gn.x + gn.y * gn.y) <= tol_abs[b] * tol_abs[b]) ? 1 : 0;
                    S.ctl[b][1] = (hn[b] == T(0)) ? 1 : 0;
                }
                __syncwarp();
            }
            if (!flow) cluster_wait();
            __syncthreads();
            for (int b = 0; b < 2; ++b) {
                if (!cact[b]) continue;
                ++iters[b];
                conv[b] = S.ctl[b][0];
                if (S.ctl[b][0] | S.ctl[b][1]) {
                    cact[b] = 0;
                    jj[b] = j + 1;
                }
            }
        }
        if (flow) flow_wait(2);  // the staging of the last step, which no apply reads
        // ---- finish the cycle of each active right-hand side ----
        if (warp < 2 && act[warp])  // back substitution of right-hand side b by warp b
            back_subst_warp<T>(S.st[warp].Rm, S.st[warp].g, S.st[warp].d, jj[warp], lane);
        __syncthreads();
        for (int t = tid; t < 2 * (MSMAX + 1); t += nt) {
            const int b = t / (MSMAX + 1), i = t - b * (MSMAX + 1);
            if (!act[b] || i > jj[b]) continue;
            Z acc = S.st[b].c[i];
            for (int l = 0; l < jj[b]; ++l) acc = cfms_<T>(S.st[b].H[i + LD * l], S.st[b].d[l], acc);
            S.st[b].rho[i] = acc;
        }
        __syncthreads();
        for (int e = tid; e < 2 * nrows; e += nt) {
            const int b = e / nrows, rr = e - b * nrows;
            if (!act[b]) continue;
            xl[b][rr] = accum_rows<T, false>(xl[b][rr], Vb[b], ldv, rr, S.st[b].d, jj[b]);
            rl[b][rr] = accum_rows<T, false>(mk<T>(0, 0), Vb[b], ldv, rr, S.st[b].rho, jj[b] + 1);
        }
        ++cycles;
        __syncthreads();
    }
    __syncthreads();
    if (flow && tid == 0 && S.fault) atomicAdd(reinterpret_cast<unsigned long long*>(&a0.out->timeouts), 1ULL);
    if (rank == 0 && tid == 0) {
        CoopStats* const outs[2] = {a0.out, a1.out};
        for (int q = 0; q < 2; ++q) {
            CoopStats* o = outs[q];
            o->ctas = ncta;
            o->spc = a0.spc;
            o->flow = flow ? 1 : 0;
            o->dc = 0;
            o->ash = 0;
            o->half = a0.Ah ? 1 : 0;
            o->paired = 1;
            o->mma = 0;
        }
        a0.out->iters += iters[0];
        a0.out->cycles += cycles;
        a0.out->solves += 1;
        a0.out->unconverged += conv[0] ? 0 : 1;
        a1.out->iters += iters[1];
        a1.out->cycles += cycles;
        a1.out->solves += 1;
        a1.out->unconverged += conv[1] ? 0 : 1;
    }
    cluster.sync();  // no CTA leaves while others may still write its shared memory
}

struct Geometry {
    int cluster = 1, spc = 1, threads = 32, vs = 0, lsw = 0, ash = 0;
    size_t smem = 0, smem_ash = 0;  // dynamic shared memory without / with the shared FP16 blocks
};

template <typename T>
mg_status geometry_uncached(long nsite, int ms, int k, int dev, Geometry& g) {
    static bool configured[2][16] = {};
    const int pi = std::is_same<T, float>::value ? 0 : 1;
    if (!configured[pi][dev]) {
        MG_CUDA_TRY(cudaFuncSetAttribute(k_coarse_proj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_LIMIT));
        MG_CUDA_TRY(cudaFuncSetAttribute(k_coarse_proj<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        configured[pi][dev] = true;
    }
    // the largest cluster (<= 16 CTAs) that can be resident; the basis slice in
    // shared memory when it fits
    for (int cl = 16; cl >= 1; cl >>= 1) {
        const long spc = (nsite + cl - 1) / cl;
        const int ctas = (int)((nsite + spc - 1) / spc);
        const int rows = (int)spc * NDOF;
        int threads = ((rows + 31) / 32) * 32;
        threads = std::min(std::max(threads, 64), MAX_THREADS);
        for (int vs = 1; vs >= 0; --vs) {
            const size_t smem = sizeof(ClusterSmem<T>) + (vs ? slice_bytes<T>(ms, rows) : 0) + proj_bytes<T>(k);
            if (smem > SMEM_LIMIT) continue;
            // push mode (basis in shared memory, one staging chunk) gets the extra
            // least-squares warp
            const int lsw = (vs && spc <= MAX_SPC) ? 1 : 0;
            const int thr = threads + 32 * lsw;
            cudaLaunchConfig_t cfg{};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = ctas;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(ctas);
            cfg.blockDim = dim3(thr);
            cfg.dynamicSmemBytes = smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_proj<T>, &cfg) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;
            }
            if (nclusters < 1) continue;
            g.cluster = ctas;
            g.spc = (int)spc;
            g.threads = thr;
            g.vs = vs;
            g.lsw = lsw;
            g.smem = smem;
            // FP32 push mode: room for the shared FP16 blocks (used when the handle
            // streams the FP16 operator), if the number of resident clusters holds
            const size_t ash_bytes = (size_t)spc * ASH_SITE_WORDS * sizeof(unsigned);
            if (std::is_same<T, float>::value && lsw && smem + ash_bytes <= SMEM_LIMIT) {
                cfg.dynamicSmemBytes = smem + ash_bytes;
                int nc2 = 0;
                if (cudaOccupancyMaxActiveClusters(&nc2, k_coarse_proj<T>, &cfg) == cudaSuccess && nc2 >= nclusters) {
                    g.ash = 1;
                    g.smem_ash = smem + ash_bytes;
                }
                (void)cudaGetLastError();
            }
            return MG_OK;
        }
    }
    set_error("coarse solve: no resident cluster shape for %ld coarse sites", nsite);
    return MG_EINVAL;
}

// geometry_uncached per (precision, device, coarse sites, ms, k), computed once
// (its occupancy queries cost host time before every coarse solve otherwise)
template <typename T>
mg_status geometry(long nsite, int ms, int k, Geometry& g) {
    struct Entry {
        long nsite;
        int ms, k, dev;
        Geometry g;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 16) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.nsite == nsite && e.ms == ms && e.k == k && e.dev == dev) {
            g = e.g;
            return MG_OK;
        }
    MG_TRY(geometry_uncached<T>(nsite, ms, k, dev, g));
    cache.push_back(Entry{nsite, ms, k, dev, g});
    return MG_OK;
}

}  // namespace

template <typename T>
mg_status launch_coarse_proj(const CoopArgs<T>& args_in, cudaStream_t s) {
    CoopArgs<T> a = args_in;
    if (a.ms < 1 || a.ms > MSMAX || a.k < 1 || a.k + 1 > PSTR || a.ms + 2 > PSTR) {
        set_error("coarse solve: unsupported (m - k, k) = (%d, %d)", a.ms, a.k);
        return MG_EINVAL;
    }
    Geometry g;
    MG_TRY(geometry<T>((long)a.Nx * a.Nt, a.ms, a.k, g));
    a.spc = g.spc;
    a.vs = g.vs;
    a.lsw = g.lsw;
    a.flow = g.lsw;  // push mode
    a.ash = (g.ash && a.Ah) ? 1 : 0;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(g.cluster);
    cfg.blockDim = dim3(g.threads);
    cfg.dynamicSmemBytes = a.ash ? g.smem_ash : g.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_coarse_proj<T>, a));
    count_launch();
    return MG_OK;
}

template mg_status launch_coarse_proj<double>(const CoopArgs<double>&, cudaStream_t);
template mg_status launch_coarse_proj<float>(const CoopArgs<float>&, cudaStream_t);

mg_status launch_coarse_proj_pair(const CoopArgs<float>& a0in, const CoopArgs<float>& a1in, cudaStream_t s,
                                  bool* launched) {
    *launched = false;
    CoopArgs<float> a0 = a0in, a1 = a1in;
    if (a0.A != a1.A || a0.Ah != a1.Ah || a0.W != a1.W || a0.pls != a1.pls || a0.k != a1.k || a0.ms != a1.ms || a0.Nx != a1.Nx ||
        a0.Nt != a1.Nt || a0.max_cycles != a1.max_cycles) {
        set_error("coarse pair solve: the two solves must share the operator and the deflation space");
        return MG_EINVAL;
    }
    if (a0.ms < 1 || a0.ms > MSMAX || a0.k < 1 || a0.k + 1 > PSTR || a0.ms + 2 > PSTR) {
        set_error("coarse pair solve: unsupported (m - k, k) = (%d, %d)", a0.ms, a0.k);
        return MG_EINVAL;
    }
    static bool configured[16] = {};
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 16) dev = 0;
    if (!configured[dev]) {
        MG_CUDA_TRY(cudaFuncSetAttribute(k_coarse_proj_pair<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_LIMIT));
        MG_CUDA_TRY(
            cudaFuncSetAttribute(k_coarse_proj_pair<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        configured[dev] = true;
    }
    // push mode only: both basis slices in shared memory, one staging chunk;
    // otherwise the caller runs the two solves one after the other
    const long nsite = (long)a0.Nx * a0.Nt;
    for (int cl = 16; cl >= 1; cl >>= 1) {
        const long spc = (nsite + cl - 1) / cl;
        if (spc > MAX_SPC) return MG_OK;
        const int ctas = (int)((nsite + spc - 1) / spc);
        const int rows = (int)spc * NDOF;
        const int threads = std::min(std::max(((rows + 31) / 32) * 32, 64), MAX_THREADS);
        const size_t smem = sizeof(PairSmem<float>) + 2 * slice_bytes<float>(a0.ms, rows) + proj_bytes<float>(a0.k);
        if (smem > SMEM_LIMIT) return MG_OK;
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ctas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(ctas);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_proj_pair<float>, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (nclusters < 1) continue;
        a0.spc = a1.spc = (int)spc;
        a0.vs = a1.vs = 1;
        a0.lsw = a1.lsw = 0;
        a0.ash = a1.ash = 0;
        a0.flow = a1.flow = 1;
        MG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_coarse_proj_pair<float>, a0, a1));
        count_launch();
        *launched = true;
        return MG_OK;
    }
    return MG_OK;
}

}  // namespace mg
