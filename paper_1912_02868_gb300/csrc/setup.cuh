// Launchers of the hierarchy set-up kernels.
#pragma once
#include "ops.cuh"

namespace mg {

// Q[B][c][j][l][a] from 12 globally orthonormal vectors V (rows, stride ldv) on a
// NxF x NtF grid with 2h dofs per site; *err = 1 on a rank-deficient block.
void launch_local_orth(double2* Q, const double2* V, long ldv, int NxF, int NtF, int h, double rank_tol, int* err,
                       cudaStream_t s);
// Galerkin stencil (column-major 24x24 blocks) of P^+ D P for the fine Wilson operator
void launch_galerkin_wilson(double2* Ac, const double2* U, double m0, const double2* Q, int Lx, int Lt,
                            cudaStream_t s);
// ... and of P^+ A P for an intermediate-grid stencil A
void launch_galerkin_stencil(double2* Ac, const double2* A, const double2* Q, int NxF, int NtF, cudaStream_t s);

}  // namespace mg
