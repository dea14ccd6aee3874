// Device-side pieces of the Krylov least squares shared by the kernels that
// update it (dense.cu, and the fused coarse block steps in coarse_block.cu):
// complex Givens rotations and the incremental push of one Arnoldi column.
#pragma once
#include "kstate.cuh"

namespace mg {
namespace ksd {

__device__ __forceinline__ double cabsd(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }
__device__ __forceinline__ double cabs2d(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabs1d(double2 a) { return fabs(a.x) + fabs(a.y); }
// a / b = a conj(b) / |b|^2 with one real reciprocal: FP64 divides and square
// roots are long dependent sequences at this GPU's FP64 rate, and these sit on
// serial paths.  (The entries here are O(1e-16..1e2), far from overflow.)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double inv = 1.0 / cabs2d(b);
    return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 z0() { return make_double2(0.0, 0.0); }

// Complex Givens rotation G = [[c, s], [-conj(s), c]] with G [a; b] = [r; 0].
// (reciprocal square roots only, no divide)
__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
    const double ab2 = cabs2d(b);
    if (ab2 == 0.0) {
        c = 1.0;
        s = z0();
        r = a;
        return;
    }
    const double aa2 = cabs2d(a);
    if (aa2 == 0.0) {
        const double inv_ab = rsqrt(ab2);
        c = 0.0;
        s = make_double2(b.x * inv_ab, -b.y * inv_ab);
        r = make_double2(ab2 * inv_ab, 0.0);
        return;
    }
    const double rho2 = aa2 + ab2;
    const double inv_aa = rsqrt(aa2), inv_rho = rsqrt(rho2);
    c = aa2 * inv_aa * inv_rho;
    const double2 ph = make_double2(a.x * inv_aa, a.y * inv_aa);
    s = cscale(cmul(ph, conj_(b)), inv_rho);
    r = cscale(ph, rho2 * inv_rho);
}
__device__ __forceinline__ void rot_apply(double c, double2 s, double2& up, double2& uq) {
    const double2 p = up, q = uq;
    up = cadd(cscale(p, c), cmul(s, q));
    uq = csub(cscale(q, c), cmul(conj_(s), p));
}

// Column jh of the Arnoldi matrix from hA + hB and sqrt(hn2): store it, apply the
// earlier rotations, add the new one, update the rotated right-hand side, the
// residual estimate, the stop flags and the gates of the next step.
__device__ inline void ks_push_dev(KState* ks, int jh) {
    if (ks->step_gate != jh) return;
    const int j = jh;
    double2* Hc = ks->H + KLD * j;
    double2* Rc = ks->R + KLD * j;
    for (int i = 0; i <= j; ++i) {
        const double2 h = cadd(ks->hA[i], ks->hB[i]);
        Hc[i] = h;
        Rc[i] = h;
    }
    for (int i = j + 2; i < KLD; ++i) {
        Hc[i] = z0();
        Rc[i] = z0();
    }
    const double hn = sqrt(fmax(ks->hn2, 0.0));
    Hc[j + 1] = make_double2(hn, 0.0);
    Rc[j + 1] = Hc[j + 1];
    const int nr = ks->nrot;
    for (int t = 0; t < nr; ++t) rot_apply(ks->rc[t], ks->rs[t], Rc[ks->ra[t]], Rc[ks->rb[t]]);
    double c;
    double2 s, r;
    givens(Rc[j], Rc[j + 1], c, s, r);
    Rc[j] = r;
    Rc[j + 1] = z0();
    ks->rc[nr] = c;
    ks->rs[nr] = s;
    ks->ra[nr] = (short)j;
    ks->rb[nr] = (short)(j + 1);
    ks->nrot = nr + 1;
    rot_apply(c, s, ks->g[j], ks->g[j + 1]);
    ks->res = cabsd(ks->g[j + 1]);
    ks->j = j + 1;
    ks->breakdown = (hn == 0.0) ? 1 : 0;
    ks->conv = (ks->res <= ks->tol_abs) ? 1 : 0;
    ks->step_gate = (ks->conv || ks->breakdown || j + 1 >= KMAX) ? -1 : j + 1;
    ks->scale_gate = (hn > 0.0) ? j + 1 : -1;
    ks->scale = (hn > 0.0) ? 1.0 / hn : 0.0;
}

}  // namespace ksd
}  // namespace mg
