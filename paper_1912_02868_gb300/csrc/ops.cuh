// Launchers of every kernel of the solve path.  Each kernel file instantiates
// its templates for T = double and T = float.
#pragma once
#include "common.cuh"

namespace mg {

// A kernel with a gate runs only when ptr == nullptr or *ptr == val.  Krylov
// cycles are enqueued whole; the gates make the steps after convergence no-ops
// without a host round trip.
//
// Batched kernels (many right-hand sides in lockstep) read the gate of
// right-hand side r at ptr[r * stride].
struct Gate {
    const int* ptr = nullptr;
    int val = 0;
    long stride = 0;
};
__device__ __forceinline__ bool gate_open(const Gate& g) { return g.ptr == nullptr || *g.ptr == g.val; }
__device__ __forceinline__ bool gate_open(const Gate& g, int r) {
    return g.ptr == nullptr || g.ptr[(long)r * g.stride] == g.val;
}

// Deterministic reductions: per-block partial sums, the last block to finish
// adds them in block order.  One workspace per stream.
constexpr int RED_THREADS = 256;
constexpr int RED_MAXD = 64;
struct RedWS {
    double2* partial = nullptr;  // [max_blocks][RED_MAXD]
    unsigned* ticket = nullptr;
    int max_blocks = 0;
};

// Launch shapes.  The level applies below take a `shape`: 0 is the built-in
// choice; otherwise threads per block (Wilson, one thread per site), WILSON_TILE + r
// (Wilson, tiles of 32 x r sites staged in shared memory), WILSON_COLS + r (Wilson,
// columns of r sites a lane in registers, x neighbours by warp shuffles), or sites
// per block (FP32 stencils).  A shape only groups sites into blocks: the arithmetic of every site,
// and so every result bit, is the same for all of them (tune.cu picks one by
// timing).
constexpr int WILSON_TILE = 1000;
constexpr int WILSON_COLS = 2000;
constexpr int WILSON_SHAPES[] = {64, 128, 256, WILSON_TILE + 4, WILSON_TILE + 8, WILSON_COLS + 2, WILSON_COLS + 4};
constexpr int STENCIL_F32_SHAPES[] = {4, 8, 16, 24, 32};
constexpr int STENCIL_LR_F32_SHAPES[] = {4, 8, 12, 16};

// ---------------------------------------------------------------- wilson ----
// y = D x, D^+ x (dagger), or y = b - D x when b != nullptr.  Section 2.
template <typename T>
void launch_wilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt,
                   bool dagger, Gate g, cudaStream_t s, int shape = 0);

// --------------------------------------------------------------- stencil ----
// y = A x (or sigma3^ A sigma3^ x, or b - A x) for the 5-point block stencil with
// dof x dof blocks stored column-major: A[s][d][l][k] is entry (k, l).
template <typename T>
void launch_stencil(C2<T>* y, const C2<T>* x, const C2<T>* A, const C2<T>* b, int Nx, int Nt, int dof,
                    bool dagger, Gate g, cudaStream_t s, int shape = 0);

// The 24-dof stencil with low-rank hop blocks (intermediate grid): per site
// LR_SITE complex entries, the self block column-major (576), then for each hop
// direction d = 1..4 the factors of A[s][d] = Q R: Q as [i][k] (4 x 24, its
// columns contiguous) and R as [i][l] (4 x 24, its rows contiguous).
constexpr int LR_RANK = 4;
constexpr int LR_SITE = 24 * 24 + 4 * 2 * LR_RANK * 24;
template <typename T>
void launch_stencil_lr(C2<T>* y, const C2<T>* x, const C2<T>* F, const C2<T>* b, int Nx, int Nt, bool dagger,
                       Gate g, cudaStream_t s, int shape = 0);
// F (FP64, LR_SITE per site) from the dense stencil A: the self blocks copied,
// each hop block factored by Gram-Schmidt with column pivoting (4 steps);
// *maxerr (device) receives max over blocks of ||A - Q R||_F / ||A||_F
void launch_factor_hops(double2* F, const double2* A, long nsite, double* maxerr, cudaStream_t s);

// -------------------------------------------------------------- transfer ----
// Q[B][c][j][l][a]: block B of the finer grid (NxF x NtF sites, 2h dofs per site),
// chirality c, vector j < 12, site l = lx + 4 lt in the block, dof a < h.
template <typename T>
void launch_restrict(C2<T>* coarse, const C2<T>* fine, const C2<T>* Q, int NxF, int NtF, int h, Gate g,
                     cudaStream_t s);
template <typename T>
void launch_prolong(C2<T>* fine, const C2<T>* coarse, const C2<T>* Q, int NxF, int NtF, int h, bool accumulate,
                    Gate g, cudaStream_t s);

// ------------------------------------------------------------------ blas ----
// out[i] = sum_e conj(V[i][e]) w[e], i < nd (rows of V have stride ldv)
template <typename T>
void launch_gram(double2* out, const C2<T>* V, long ldv, int nd, const C2<T>* w, long n, RedWS ws, Gate g,
                 cudaStream_t s);
// w[e] = (zero_first ? 0 : w[e]) + sign * sum_i V[i][e] coef[i], i < count,
// count = nd_dev ? *nd_dev + nd : nd.  If norm2_out: *norm2_out = ||w||^2 after.
template <typename T>
void launch_axpy_multi(C2<T>* w, const C2<T>* V, long ldv, int nd, const int* nd_dev, const double2* coef,
                       double sign, bool zero_first, long n, double* norm2_out, RedWS ws, Gate g, cudaStream_t s);
template <typename T>
void launch_norm2(double* out, const C2<T>* v, long n, RedWS ws, Gate g, cudaStream_t s);
// y = x * (*factor)
template <typename T>
void launch_scale(C2<T>* y, const C2<T>* x, const double* factor, long n, Gate g, cudaStream_t s);
// y = x (precision change)
template <typename Ta, typename Tb>
void launch_convert(C2<Tb>* y, const C2<Ta>* x, long n, Gate g, cudaStream_t s);
// y = x + a * y  with a = (*num / *den) (CG search direction update), or when
// den == nullptr, a = *num.
// FP16 copy of a complex FP64 array: y[i] = half(re) | half(im) << 16
void launch_pack_half(unsigned* y, const double2* x, long n, cudaStream_t s);
template <typename T>
void launch_xpay(C2<T>* y, const C2<T>* x, const double* num, const double* den, long n, Gate g, cudaStream_t s);
// CG step: e += alpha p, r -= alpha q, alpha = *rr / *pq (real); *rr_new = ||r||^2
template <typename T>
void launch_cg_step(C2<T>* e, C2<T>* r, const C2<T>* p, const C2<T>* q, const double* rr, const double* pq,
                    double* rr_new, long n, RedWS ws, Gate g, cudaStream_t s);
// *out = Re <x, y>
template <typename T>
void launch_redot(double* out, const C2<T>* x, const C2<T>* y, long n, RedWS ws, Gate g, cudaStream_t s);

}  // namespace mg
