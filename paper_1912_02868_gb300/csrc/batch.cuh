// Kernels of the lockstep multi-right-hand-side solve: vectors of a block of
// right-hand sides are stored RHS-major (right-hand side r at base + r * stride),
// every kernel runs all of them in one launch, and per-right-hand-side gates
// (Gate with a stride) switch individual right-hand sides off.
#pragma once
#include "ops.cuh"

namespace mg {

constexpr int NB_MAX = 64;   // right-hand sides of one block
constexpr int NB_TILE = 8;   // right-hand sides of one tensor-core tile (MMA n = 8)

// per-right-hand-side reduction workspace: partial[r][chunk][RED_MAXD], ticket[r]
struct BRed {
    double2* partial = nullptr;  // NB_MAX * max_chunks * RED_MAXD entries (read as C2<T>)
    unsigned* ticket = nullptr;  // NB_MAX
    int max_chunks = 0;
};

// out[r*os + i] = sum_e conj(V[r*vr + i*ldv + e]) w[r*wr + e], i < nd + (ndd ? ndd[r*nds] : 0)
template <typename T>
void launch_bgram(double2* out, long os, const C2<T>* V, long ldv, long vr, int nd, const int* ndd, long nds,
                  const C2<T>* w, long wr, long n, int nb, BRed red, Gate g, cudaStream_t s);
// w[r] = (zero_first ? 0 : w[r]) + sign sum_i V[r][i] coef[r*cs + i]; optionally
// norm2[r*n2s] = ||w[r]||^2 after
template <typename T>
void launch_baxpy(C2<T>* w, long wr, const C2<T>* V, long ldv, long vr, int nd, const int* ndd, long nds,
                  const double2* coef, long cs, double sign, bool zero_first, long n, int nb, double* norm2,
                  long n2s, BRed red, Gate g, cudaStream_t s);
template <typename T>
void launch_bnorm2(double* out, long os, const C2<T>* v, long vr, long n, int nb, BRed red, Gate g, cudaStream_t s);
// y[r] = x[r] * f[r*fs]
template <typename T>
void launch_bscale(C2<T>* y, long yr, const C2<T>* x, long xr, const double* f, long fs, long n, int nb, Gate g,
                   cudaStream_t s);
// y[r] = x[r] (precision change), n entries per right-hand side, all right-hand sides
template <typename Ta, typename Tb>
void launch_bconvert(C2<Tb>* y, long yr, const C2<Ta>* x, long xr, long n, int nb, cudaStream_t s);

// Wilson-Dirac apply / residual for every right-hand side (vectors of n0 = 2 Lx Lt)
template <typename T>
void launch_bwilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt, long vr,
                    int nb, Gate g, cudaStream_t s);
template <typename T>
void launch_brestrict(C2<T>* coarse, long cr, const C2<T>* fine, long fr, const C2<T>* Q, int NxF, int NtF, int h,
                      int nb, Gate g, cudaStream_t s);
template <typename T>
void launch_bprolong(C2<T>* fine, long fr, const C2<T>* coarse, long cr, const C2<T>* Q, int NxF, int NtF, int h,
                     bool accumulate, int nb, Gate g, cudaStream_t s);

// Operator of a 24-dof block stencil for the tensor-core apply: every 8 x 8
// complex tile (output rows 8 mt.., input columns 8 kt..) of every block A[s][d]
// as 64 words (16-bit real part in the low half, imaginary in the high half,
// BF16 or FP16, each rounded once from FP64) in the order the MMA fragments load
// them.  4 * 5 * 576 bytes per site.
void launch_pack_frag(unsigned* out, const double2* A, long nsite, bool fp16, cudaStream_t s);

// Y[r] = A X[r] (or B[r] - A X[r]) for the block of nb right-hand sides (nb a
// multiple of 8): the 24 x 24 complex block products on tensor cores
// (mma.sync m16n8k16, BF16 or FP16 inputs, FP32 accumulation), each complex
// product as one real 48 x 48 product; the FP32 vector is split into a high and
// a low 16-bit part so that only the operator is rounded.  Right-hand sides
// with a closed gate are not written.
void launch_bstencil_mma(float2* Y, const float2* X, const float2* B, long vr, const unsigned* Af, int Nx, int Nt,
                         int nb, bool fp16, Gate g, cudaStream_t s);

}  // namespace mg
