// Device-resident state of one Krylov cycle (FP64): the Arnoldi matrix, its
// QR factorisation by Givens rotations, the least-squares right-hand side, and
// the gates that let a whole cycle be enqueued without host round trips.
#pragma once
#include <cstddef>
#include <type_traits>

#include "ops.cuh"

namespace mg {

constexpr int KMAX = 48;          // largest Krylov dimension m (GMRES-DR(40,16) needs 40)
constexpr int KLD = KMAX + 1;     // leading dimension: column-major H[i + KLD * j]
constexpr int NROT = KMAX * (KMAX + 1) / 2 + KMAX + 8;

struct alignas(16) KState {
    double2 H[KLD * KMAX];   // Arnoldi matrix as built (unrotated)
    double2 R[KLD * KMAX];   // rotated: upper triangular in columns < j
    double2 c[KLD];          // least-squares right-hand side (unrotated)
    double2 g[KLD];          // rotated right-hand side
    double2 hA[KLD], hB[KLD];// the two Gram passes of CGS2 for the current column
    double2 d[KMAX];         // least-squares solution (after finish)
    double2 rho[KLD];        // c - H d (after finish)
    double2 u[KLD];          // scratch
    double rc[NROT];         // rotations in the order applied: rows (ra, rb), cos, sin
    double2 rs[NROT];
    short ra[NROT], rb[NROT];
    double hn2;              // ||w||^2 after orthogonalisation
    double scale;            // factor of the next basis vector (1/h or 1/beta)
    double beta;             // norm of the starting residual
    double tol_abs;          // stop when the least-squares residual <= tol_abs
    double res;              // current least-squares residual norm
    int nrot;
    int j, j0;               // columns built; first column of this cycle
    int step_gate;           // = j while the cycle continues, -1 once stopped
    int scale_gate;          // = j after a push whose new vector is normalisable
    int conv, breakdown, err;
};

// Output of a GMRES-DR restart: the (j+1) x (k+1) matrix P_{k+1}, the new
// (k+1) x k Hessenberg block H_k = P^+ H P_k and c = P^+ rho (Morgan 2002).
struct DRState {
    double2 P[KLD * (KMAX + 1)];
    double2 Hk[KLD * KMAX];
    double2 ck[KLD];
    double2 theta[KMAX];     // harmonic Ritz values, ascending |theta|
    int j, k, err;
};

// Start a cycle from a vector of squared norm *nrm2: beta = sqrt(*nrm2),
// stop when the least-squares residual <= tol_rel * sqrt(*nb2).
void ks_start(KState* ks, const double* nrm2, double tol_rel, const double* nb2, cudaStream_t s);
void ks_push(KState* ks, int jh, cudaStream_t s);
void ks_finish(KState* ks, cudaStream_t s);
// Load a dense (k+1) x k block H_k and c (k+1) (column-major, ld KLD) and
// factor it: the next cycle continues the Arnoldi process from column k.
// ck == nullptr means c = 0; tol_abs < 0 keeps the state's tolerance.
void ks_load_dense(KState* ks, const double2* Hk, const double2* ck, int k, double tol_abs, cudaStream_t s);
// GMRES-Proj least squares with a prepared (ks_load_dense) state:
// d = argmin ||cvec - H_k d||, u = H_k d.
void proj_solve(const KState* pls, const double2* cvec, double2* d, double2* u, cudaStream_t s);
// Batched forms over the states ks[0..nb): per right-hand side r the scalars
// at nrm2[r * ns], nb2[r * nbs], cvec[r * cs], ...; bks_start starts a closed
// gate's right-hand side as an empty cycle (converged, no steps).
void bks_start(KState* ks, int nb, const double* nrm2, long ns, double tol_rel, const double* nb2, long nbs, Gate act,
               cudaStream_t s);
void bks_push(KState* ks, int nb, int jh, cudaStream_t s);
void bks_finish(KState* ks, int nb, cudaStream_t s);
void bproj_solve(const KState* pls, int nb, const double2* cvec, long cs, double2* d, long ds, double2* u, long us,
                 Gate act, cudaStream_t s);
// strides of KState fields across an array of states, in units of the field's type
static_assert(sizeof(KState) % sizeof(double2) == 0, "KState arrays are strided in whole double2 units");
constexpr long KS_INTS = (long)(sizeof(KState) / sizeof(int));
constexpr long KS_DBLS = (long)(sizeof(KState) / sizeof(double));
constexpr long KS_CPLX = (long)(sizeof(KState) / sizeof(double2));

// GMRES-DR restart from the finished cycle in ks (harmonic Ritz vectors).
mg_status dr_restart(const KState* ks, DRState* dr, int k, cudaStream_t s);
// *out = 1 / sqrt(*in)
void scalar_rsqrt(double* out, const double* in, cudaStream_t s);
// *out = v
void scalar_set(double* out, double v, cudaStream_t s);
// CG bookkeeping: start (rr = nb2 = *r2, active = rr > tol^2 nb2) and, after
// each step while active, rr = rr_new, iters += 1, active = rr_new > tol^2 nb2.
void cg_init(const double* r2, double* rr, double* nb2, double tol, int* active, int* iters, cudaStream_t s);
void cg_scalars(double* rr, const double* rr_new, const double* nb2, double tol, int* active, int* iters,
                cudaStream_t s);

// address of a field of a struct that lives in device memory
#define MG_DEVF(ptr, type, field)                          \
    reinterpret_cast<type*>(reinterpret_cast<char*>(ptr) + \
                            offsetof(std::remove_pointer_t<decltype(ptr)>, field))

}  // namespace mg
