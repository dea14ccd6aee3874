// Fine-grid Wilson-Dirac operator of the 2D Schwinger model (Section 2):
//
//   (D psi)(s) = (m0 + 2) psi(s)
//              - 1/2 sum_mu [ (1 - sigma_mu) U_mu(s) psi(s + mu)
//                           + (1 + sigma_mu) U_mu(s - mu)^* psi(s - mu) ]
//
// sigma_1 on x, sigma_2 on t, periodic in x, antiperiodic in t (a hop across
// t = L_t - 1 <-> 0 carries -1).  D^+ = sigma_3 D sigma_3.
//
// Each (1 -/+ sigma_mu) has rank one, so a hop moves one complex number h:
//   +x: h = U_x(s)   (p0 - p1),        contributes (-h/2, +h/2)
//   -x: h = U_x^*(s-x)(p0 + p1),       contributes (-h/2, -h/2)
//   +t: h = U_t(s)   (p0 + i p1),      contributes (-h/2, +i h/2)
//   -t: h = U_t^*(s-t)(p0 - i p1),     contributes (-h/2, -i h/2)
// Three launch forms with the same per-site arithmetic (wilson_site), so the
// same result bits:
// * k_wilson: one thread per site; the site's two spin components and its two
//   links are one 32-byte (FP64) or 16-byte (FP32) vector load each.  Neighbour
//   spinors are re-read by four threads and come from L1/L2.
// * k_wilson_tile: a block owns a tile of 32 x TY sites and stages, with
//   coalesced row loads, the spinors of the tile and a one-site halo and the
//   links of the tile with the column to its left and the row below in shared
//   memory; each thread then reads its five spinors and three links there.
//   Every spinor and link comes from global memory once per tile (plus the
//   halo: (TY + 2)(34) spinors and (TY + 1)(33) link pairs for 32 TY sites).
// * k_wilson_col: a warp owns 32 columns of R sites along t; each lane keeps
//   its column's R + 2 spinors and R + 1 link pairs in registers (one coalesced
//   row load each) and takes its x neighbours from the adjacent lanes by warp
//   shuffles, so a site costs about (2R + 3) / R loads instead of eight, all
//   independent, with no barrier.  Lanes whose neighbour is not the adjacent
//   lane's site (the warp's edge lanes, the periodic wrap) load it directly.
#include "batch.cuh"

namespace mg {

namespace {

template <typename T> struct alignas(2 * sizeof(C2<T>)) Pair {
    C2<T> a, b;
};

template <typename T, bool DAG>
__device__ __forceinline__ void spins(const Pair<T>& v, C2<T>& p0, C2<T>& p1) {
    p0 = v.a;
    p1 = DAG ? cneg(v.b) : v.b;
}

// Explicitly rounded operations for the site arithmetic: the compiler may not
// fuse or reorder them, so every launch form of the apply (each inlines
// wilson_site into a different loop) rounds identically, bit for bit.
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename Z> __device__ __forceinline__ Z z_add(Z a, Z b) {
    a.x = r_add(a.x, b.x);
    a.y = r_add(a.y, b.y);
    return a;
}
template <typename Z> __device__ __forceinline__ Z z_sub(Z a, Z b) { return z_add(a, cneg(b)); }
// a * b
template <typename Z> __device__ __forceinline__ Z z_mul(Z a, Z b) {
    Z c;
    c.x = r_fma(a.x, b.x, -r_mul(a.y, b.y));
    c.y = r_fma(a.x, b.y, r_mul(a.y, b.x));
    return c;
}
// conj(a) * b
template <typename Z> __device__ __forceinline__ Z z_mulc(Z a, Z b) {
    Z c;
    c.x = r_fma(a.x, b.x, r_mul(a.y, b.y));
    c.y = r_fma(a.x, b.y, -r_mul(a.y, b.x));
    return c;
}

// One site of y = D x (D^+ x with DAG, b - D x with RES) from its loaded
// operands: the spinors of the site (vs) and of its four neighbours, the site's
// links us = (U_x(s), U_t(s)), U_x(s - x), U_t(s - t), and the signs of the
// forward (sf) and backward (sb) t hops (-1 across the antiperiodic boundary).
template <typename T, bool DAG, bool RES>
__device__ __forceinline__ Pair<T> wilson_site(const Pair<T>& vs, const Pair<T>& vxp, const Pair<T>& vxm,
                                               const Pair<T>& vtp, const Pair<T>& vtm, const Pair<T>& us,
                                               const C2<T>& uxm, const C2<T>& utm, T sf, T sb, T diag,
                                               const Pair<T>& bb) {
    C2<T> p0, p1, q0, q1;
    spins<T, DAG>(vs, p0, p1);
    // sum of the hops before the factor -1/2: spin 0 and spin 1 parts
    C2<T> a0, a1, h;
    // +x
    spins<T, DAG>(vxp, q0, q1);
    h = z_mul(us.a, z_sub(q0, q1));
    a0 = h;
    a1 = cneg(h);
    // -x
    spins<T, DAG>(vxm, q0, q1);
    h = z_mulc(uxm, z_add(q0, q1));
    a0 = z_add(a0, h);
    a1 = z_add(a1, h);
    // +t
    spins<T, DAG>(vtp, q0, q1);
    h = z_mul(us.b, z_add(q0, cmuli(q1)));
    if (sf < T(0)) h = cneg(h);
    a0 = z_add(a0, h);
    a1 = z_sub(a1, cmuli(h));
    // -t
    spins<T, DAG>(vtm, q0, q1);
    h = z_mulc(utm, z_sub(q0, cmuli(q1)));
    if (sb < T(0)) h = cneg(h);
    a0 = z_add(a0, h);
    a1 = z_add(a1, cmuli(h));

    // (m0 + 2) p - a / 2, one rounding per component (a / 2 is exact)
    C2<T> o0, o1;
    o0.x = r_fma(diag, p0.x, r_mul(T(-0.5), a0.x));
    o0.y = r_fma(diag, p0.y, r_mul(T(-0.5), a0.y));
    o1.x = r_fma(diag, p1.x, r_mul(T(-0.5), a1.x));
    o1.y = r_fma(diag, p1.y, r_mul(T(-0.5), a1.y));
    if (DAG) o1 = cneg(o1);
    if (RES) {
        o0 = z_sub(bb.a, o0);
        o1 = z_sub(bb.b, o1);
    }
    Pair<T> out;
    out.a = o0;
    out.b = o1;
    return out;
}

// blockIdx.y = right-hand side r of a batch: vectors at offset r * vr, gate r
template <typename T, bool DAG, bool RES>
__global__ void __launch_bounds__(256) k_wilson(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                const C2<T>* __restrict__ U, const C2<T>* __restrict__ b,
                                                T diag, int Lx, int Lt, long vr, Gate g) {
    const int rb = blockIdx.y;
    if (!gate_open(g, rb)) return;
    y += rb * vr;
    x += rb * vr;
    if (RES) b += rb * vr;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Lx * Lt) return;
    const int xx = s % Lx, t = s / Lx;
    const int sxp = (xx + 1 == Lx) ? s - xx : s + 1;
    const int sxm = (xx == 0) ? s + Lx - 1 : s - 1;
    const int stp = (t + 1 == Lt) ? xx : s + Lx;
    const int stm = (t == 0) ? s + Lx * (Lt - 1) : s - Lx;
    const T sf = (t + 1 == Lt) ? T(-1) : T(1);
    const T sb = (t == 0) ? T(-1) : T(1);

    const Pair<T>* U2 = reinterpret_cast<const Pair<T>*>(U);
    const Pair<T>* X2 = reinterpret_cast<const Pair<T>*>(x);
    Pair<T> bb{};
    if (RES) bb = reinterpret_cast<const Pair<T>*>(b)[s];
    reinterpret_cast<Pair<T>*>(y)[s] = wilson_site<T, DAG, RES>(X2[s], X2[sxp], X2[sxm], X2[stp], X2[stm], U2[s],
                                                                U2[sxm].a, U2[stm].b, sf, sb, diag, bb);
}

// v mod n for v >= -1 (a tile or column coordinate with its one-site halo)
__device__ __forceinline__ int wrap(int v, int n) {
    if (v < 0) return v + n;
    return v < n ? v : v % n;
}

// blockDim (32, TY): a tile of 32 (x) by TY (t) sites; blockIdx.z = right-hand
// side r of a batch (vectors at offset r * vr, gate r).  Shared memory entry
// (i, j) of the spinor tile holds site ((x0 - 1 + i) mod L_x, (t0 - 1 + j) mod L_t),
// 0 <= i < 34, 0 <= j < TY + 2, and of the link tile the links of site
// ((x0 - 1 + i) mod L_x, (t0 - 1 + j) mod L_t), 0 <= i < 33, 0 <= j < TY + 1.  A
// neighbour of a site is then the adjacent entry even where the tile is ragged
// or wider than the lattice, and the wrap is the periodic boundary.
template <typename T, bool DAG, bool RES, int TY>
__global__ void __launch_bounds__(32 * TY) k_wilson_tile(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                         const C2<T>* __restrict__ U, const C2<T>* __restrict__ b,
                                                         T diag, int Lx, int Lt, long vr, Gate g) {
    constexpr int TX = 32, SW = TX + 2, UW = TX + 1, NT = TX * TY;
    __shared__ Pair<T> sx[(TY + 2) * SW];
    __shared__ Pair<T> su[(TY + 1) * UW];
    const int rb = blockIdx.z;
    if (!gate_open(g, rb)) return;  // the same for every thread of the block
    y += rb * vr;
    x += rb * vr;
    if (RES) b += rb * vr;
    const int x0 = blockIdx.x * TX, t0 = blockIdx.y * TY;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const Pair<T>* X2 = reinterpret_cast<const Pair<T>*>(x);
    const Pair<T>* U2 = reinterpret_cast<const Pair<T>*>(U);
    for (int e = tid; e < (TY + 2) * SW; e += NT) {
        const int j = e / SW, i = e - j * SW;
        sx[e] = X2[wrap(x0 - 1 + i, Lx) + (long)Lx * wrap(t0 - 1 + j, Lt)];
    }
    for (int e = tid; e < (TY + 1) * UW; e += NT) {
        const int j = e / UW, i = e - j * UW;
        su[e] = U2[wrap(x0 - 1 + i, Lx) + (long)Lx * wrap(t0 - 1 + j, Lt)];
    }
    __syncthreads();
    const int xx = x0 + (int)threadIdx.x, t = t0 + (int)threadIdx.y;
    if (xx >= Lx || t >= Lt) return;
    const long s = xx + (long)Lx * t;
    const int c = ((int)threadIdx.y + 1) * SW + (int)threadIdx.x + 1;  // the site in sx
    const int cu = ((int)threadIdx.y + 1) * UW + (int)threadIdx.x + 1;  // its links in su
    const T sf = (t + 1 == Lt) ? T(-1) : T(1);
    const T sb = (t == 0) ? T(-1) : T(1);
    Pair<T> bb{};
    if (RES) bb = reinterpret_cast<const Pair<T>*>(b)[s];
    reinterpret_cast<Pair<T>*>(y)[s] = wilson_site<T, DAG, RES>(sx[c], sx[c + 1], sx[c - 1], sx[c + SW], sx[c - SW],
                                                                su[cu], su[cu - 1].a, su[cu - UW].b, sf, sb, diag,
                                                                bb);
}

// a Pair from lane (lane + d) of the warp (d = +1 or -1); every lane takes part
template <typename T>
__device__ __forceinline__ Pair<T> shfl_pair(const Pair<T>& p, int d) {
    Pair<T> q;
    if (d > 0) {
        q.a.x = __shfl_down_sync(0xffffffffu, p.a.x, 1);
        q.a.y = __shfl_down_sync(0xffffffffu, p.a.y, 1);
        q.b.x = __shfl_down_sync(0xffffffffu, p.b.x, 1);
        q.b.y = __shfl_down_sync(0xffffffffu, p.b.y, 1);
    } else {
        q.a.x = __shfl_up_sync(0xffffffffu, p.a.x, 1);
        q.a.y = __shfl_up_sync(0xffffffffu, p.a.y, 1);
        q.b.x = __shfl_up_sync(0xffffffffu, p.b.x, 1);
        q.b.y = __shfl_up_sync(0xffffffffu, p.b.y, 1);
    }
    return q;
}

// blockDim (32, 4): warp w of block (bx, by) owns sites x = 32 bx + lane,
// t = (4 by + w) R + k, k < R; blockIdx.z = right-hand side r of a batch
// (vectors at offset r * vr, gate r).  Lanes past L_x read the last column (in
// bounds) and store nothing; sites past L_t are not stored.
template <typename T, bool DAG, bool RES, int R>
__global__ void __launch_bounds__(128) k_wilson_col(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                    const C2<T>* __restrict__ U, const C2<T>* __restrict__ b,
                                                    T diag, int Lx, int Lt, long vr, Gate g) {
    const int rb = blockIdx.z;
    if (!gate_open(g, rb)) return;  // the same for every thread of the block
    y += rb * vr;
    x += rb * vr;
    if (RES) b += rb * vr;
    const int lane = threadIdx.x;
    const int xx = blockIdx.x * 32 + lane;
    const bool live = xx < Lx;
    const int xc = live ? xx : Lx - 1;
    const int xp = (xc + 1 == Lx) ? 0 : xc + 1;
    const int xm = (xc == 0) ? Lx - 1 : xc - 1;
    // the +x (-x) neighbour is the next (previous) lane's own site
    const bool adj_p = lane < 31 && xc + 1 < Lx;
    const bool adj_m = lane > 0 && xc > 0;
    const int t0 = (blockIdx.y * 4 + threadIdx.y) * R;
    const Pair<T>* X2 = reinterpret_cast<const Pair<T>*>(x);
    const Pair<T>* U2 = reinterpret_cast<const Pair<T>*>(U);
    Pair<T> v[R + 2], u[R + 1];
    int row[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) row[k] = Lx * wrap(t0 - 1 + k, Lt);
#pragma unroll
    for (int k = 0; k < R + 2; ++k) v[k] = X2[xc + (long)row[k]];
#pragma unroll
    for (int k = 0; k < R + 1; ++k) u[k] = U2[xc + (long)row[k]];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int t = t0 + k;
        Pair<T> vp = shfl_pair(v[k + 1], +1);
        Pair<T> vm = shfl_pair(v[k + 1], -1);
        Pair<T> um = shfl_pair(u[k + 1], -1);
        if (!adj_p) vp = X2[xp + (long)row[k + 1]];
        if (!adj_m) {
            vm = X2[xm + (long)row[k + 1]];
            um = U2[xm + (long)row[k + 1]];
        }
        if (!live || t >= Lt) continue;
        const long s = xc + (long)row[k + 1];
        const T sf = (t + 1 == Lt) ? T(-1) : T(1);
        const T sb = (t == 0) ? T(-1) : T(1);
        Pair<T> bb{};
        if (RES) bb = reinterpret_cast<const Pair<T>*>(b)[s];
        reinterpret_cast<Pair<T>*>(y)[s] = wilson_site<T, DAG, RES>(v[k + 1], vp, vm, v[k + 2], v[k], u[k + 1], um.a,
                                                                    u[k].b, sf, sb, diag, bb);
    }
}

}  // namespace

// threads: threads per block, one thread per site (a multiple of 32, at most 256)
template <typename T>
void wilson_grid(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt, bool dagger,
                 long vr, int nb, Gate g, cudaStream_t s, int threads = 256) {
    const int n = Lx * Lt;
    const dim3 grid(nblocks(n, threads), nb);
    const T diag = (T)(m0 + 2.0);
    if (dagger) {
        if (b) k_wilson<T, true, true><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson<T, true, false><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    } else {
        if (b) k_wilson<T, false, true><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson<T, false, false><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    }
    count_launch();
}

// tiles of 32 x TY sites staged in shared memory (k_wilson_tile)
template <typename T, int TY>
void wilson_tile_grid(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt,
                      bool dagger, long vr, int nb, Gate g, cudaStream_t s) {
    const dim3 grid(nblocks(Lx, 32), nblocks(Lt, TY), nb);
    const dim3 block(32, TY);
    const T diag = (T)(m0 + 2.0);
    if (dagger) {
        if (b) k_wilson_tile<T, true, true, TY><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson_tile<T, true, false, TY><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    } else {
        if (b) k_wilson_tile<T, false, true, TY><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson_tile<T, false, false, TY><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    }
    count_launch();
}

// columns of R sites a lane, four warps a block (k_wilson_col)
template <typename T, int R>
void wilson_col_grid(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt,
                     bool dagger, long vr, int nb, Gate g, cudaStream_t s) {
    const dim3 grid(nblocks(Lx, 32), nblocks(Lt, 4 * R), nb);
    const dim3 block(32, 4);
    const T diag = (T)(m0 + 2.0);
    if (dagger) {
        if (b) k_wilson_col<T, true, true, R><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson_col<T, true, false, R><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    } else {
        if (b) k_wilson_col<T, false, true, R><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson_col<T, false, false, R><<<grid, block, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    }
    count_launch();
}

// shape: 0 (built-in: 256 threads a block, one site each), 64 / 128 / 256 threads a
// block, WILSON_TILE + 4 / + 8 (tiles of 32 x 4 or 32 x 8 sites in shared memory), or
// WILSON_COLS + 2 / + 4 (columns of 2 or 4 sites a lane, x neighbours by shuffles)
template <typename T>
void launch_wilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt,
                   bool dagger, Gate g, cudaStream_t s, int shape) {
    if (shape == WILSON_COLS + 2 && nblocks(Lt, 8) <= 65535u) {
        wilson_col_grid<T, 2>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s);
        return;
    }
    if (shape == WILSON_COLS + 4 && nblocks(Lt, 16) <= 65535u) {
        wilson_col_grid<T, 4>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s);
        return;
    }
    if (shape == WILSON_TILE + 4 && nblocks(Lt, 4) <= 65535u) {
        wilson_tile_grid<T, 4>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s);
        return;
    }
    if (shape == WILSON_TILE + 8 && nblocks(Lt, 8) <= 65535u) {
        wilson_tile_grid<T, 8>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s);
        return;
    }
    const int threads = (shape >= 32 && shape <= 256 && shape % 32 == 0) ? shape : 256;
    wilson_grid<T>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s, threads);
}

template <typename T>
void launch_bwilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt, long vr,
                    int nb, Gate g, cudaStream_t s) {
    wilson_grid<T>(y, x, U, b, m0, Lx, Lt, false, vr, nb, g, s);
}

template void launch_wilson<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, double,
                                    int, int, bool, Gate, cudaStream_t, int);
template void launch_wilson<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, double, int,
                                   int, bool, Gate, cudaStream_t, int);
template void launch_bwilson<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, double,
                                     int, int, long, int, Gate, cudaStream_t);
template void launch_bwilson<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, double, int,
                                    int, long, int, Gate, cudaStream_t);

}  // namespace mg
