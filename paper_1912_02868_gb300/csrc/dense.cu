// Small dense FP64 kernels of the Krylov solvers, all on the device:
//  * incremental least squares of (F)GMRES by complex Givens rotations
//    (FGMRES(8), the GMRES(2) smoother, GMRES-DR and GMRES-Proj cycles, Section 2);
//  * the GMRES-DR(m,k) restart of Morgan (2002): harmonic Ritz pairs of the
//    Arnoldi matrix, (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T) g = theta g, by a
//    one-CTA Householder-Hessenberg + shifted complex QR eigensolver, then the
//    new basis coefficients P_{k+1}, H_k = P_{k+1}^+ H P_k and c = P_{k+1}^+ rho;
//  * the GMRES-Proj minimum-residual projection onto the deflation space.
// These run once per Krylov step or restart on matrices of order <= 48.
#include "ks_dev.cuh"

namespace mg {

namespace {

using namespace ksd;

__device__ void ks_start_dev(KState* ks, double nrm2v, double tol_rel, double nb2v) {
    const double beta = sqrt(fmax(nrm2v, 0.0));
    const double tol_abs = tol_rel * sqrt(fmax(nb2v, 0.0));
    for (int i = 0; i < KLD; ++i) {
        ks->c[i] = z0();
        ks->g[i] = z0();
    }
    ks->c[0] = make_double2(beta, 0.0);
    ks->g[0] = ks->c[0];
    ks->beta = beta;
    ks->tol_abs = tol_abs;
    ks->res = beta;
    ks->nrot = 0;
    ks->j = 0;
    ks->j0 = 0;
    ks->conv = (beta <= tol_abs) ? 1 : 0;
    ks->breakdown = 0;
    ks->err = 0;
    ks->step_gate = (!ks->conv && beta > 0.0) ? 0 : -1;
    ks->scale = beta > 0.0 ? 1.0 / beta : 0.0;
    ks->scale_gate = 0;
}
__global__ void k_ks_start(KState* ks, const double* nrm2, double tol_rel, const double* nb2) {
    if (threadIdx.x != 0) return;
    ks_start_dev(ks, *nrm2, tol_rel, *nb2);
}
// right-hand side r of a batch: state ks[r], norms nrm2[r * ns] and nb2[r * nbs];
// a closed gate starts the cycle as if from a zero vector (nothing to do)
__global__ void k_bks_start(KState* ks, const double* nrm2, long ns, double tol_rel, const double* nb2, long nbs,
                            Gate act) {
    if (threadIdx.x != 0) return;
    const int r = blockIdx.x;
    const bool on = gate_open(act, r);
    ks_start_dev(ks + r, on ? nrm2[r * ns] : 0.0, tol_rel, on ? nb2[r * nbs] : 0.0);
}

__global__ void k_ks_push(KState* ks, int jh) {
    if (threadIdx.x != 0) return;
    ks_push_dev(ks, jh);
}
__global__ void k_bks_push(KState* ks, int jh) {
    if (threadIdx.x != 0) return;
    ks_push_dev(ks + blockIdx.x, jh);
}

// Back substitution R d = g over the first j columns, then rho = c - H d.
// One warp.
__device__ void solve_upper(const double2* R, const double2* g, double2* d, int jj, int* err) {
    const int lane = threadIdx.x & 31;
    for (int i = jj - 1; i >= 0; --i) {
        double2 acc = z0();
        for (int l = i + 1 + lane; l < jj; l += 32) acc = cfma(R[i + KLD * l], d[l], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const double2 piv = R[i + KLD * i];
            if (piv.x == 0.0 && piv.y == 0.0) {
                d[i] = z0();
                if (err) *err = 2;
            } else {
                d[i] = cdiv(csub(g[i], acc), piv);
            }
        }
        __syncwarp();
    }
}

__device__ void ks_finish_dev(KState* ks) {
    const int jj = ks->j;
    const int lane = threadIdx.x & 31;
    solve_upper(ks->R, ks->g, ks->d, jj, &ks->err);
    __syncwarp();
    double part = 0.0;
    for (int i = lane; i <= jj; i += 32) {
        double2 acc = ks->c[i];
        for (int l = 0; l < jj; ++l) acc = csub(acc, cmul(ks->H[i + KLD * l], ks->d[l]));
        ks->rho[i] = acc;
        part += acc.x * acc.x + acc.y * acc.y;
    }
    for (int i = jj + 1 + lane; i < KLD; i += 32) ks->rho[i] = z0();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) ks->res = sqrt(part);
}
__global__ void k_ks_finish(KState* ks) { ks_finish_dev(ks); }
__global__ void k_bks_finish(KState* ks) { ks_finish_dev(ks + blockIdx.x); }

__global__ void k_ks_load_dense(KState* ks, const double2* Hk, const double2* ck, int k, double tol_abs) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < KLD * KMAX; e += 32) {
        const int i = e % KLD, jc = e / KLD;
        const double2 v = (i <= k && jc < k) ? Hk[i + KLD * jc] : z0();
        ks->H[e] = v;
        ks->R[e] = v;
    }
    for (int i = lane; i < KLD; i += 32) {
        const double2 v = (i <= k && ck != nullptr) ? ck[i] : z0();
        ks->c[i] = v;
        ks->g[i] = v;
    }
    const double tol_keep = ks->tol_abs;
    __syncwarp();
    // QR of the dense (k+1) x k block: for column i zero rows k..i+1 bottom-up
    int nr = 0;
    for (int i = 0; i < k; ++i) {
        for (int r = k; r > i; --r) {
            double c = 1.0;
            double2 s = z0(), rr = z0();
            if (lane == 0) givens(ks->R[(r - 1) + KLD * i], ks->R[r + KLD * i], c, s, rr);
            c = __shfl_sync(0xffffffffu, c, 0);
            s.x = __shfl_sync(0xffffffffu, s.x, 0);
            s.y = __shfl_sync(0xffffffffu, s.y, 0);
            for (int col = i + lane; col < k; col += 32)
                rot_apply(c, s, ks->R[(r - 1) + KLD * col], ks->R[r + KLD * col]);
            __syncwarp();
            if (lane == 0) {
                ks->R[r + KLD * i] = z0();
                rot_apply(c, s, ks->g[r - 1], ks->g[r]);
                ks->rc[nr] = c;
                ks->rs[nr] = s;
                ks->ra[nr] = (short)(r - 1);
                ks->rb[nr] = (short)r;
            }
            ++nr;
            __syncwarp();
        }
    }
    if (lane == 0) {
        ks->nrot = nr;
        ks->res = cabsd(ks->g[k]);
        ks->beta = ks->res;
        ks->tol_abs = tol_abs < 0.0 ? tol_keep : tol_abs;
        tol_abs = ks->tol_abs;
        ks->j = k;
        ks->j0 = k;
        ks->conv = (ks->res <= tol_abs) ? 1 : 0;
        ks->breakdown = 0;
        ks->err = 0;
        ks->step_gate = ks->conv ? -1 : k;
        ks->scale_gate = -1;
        ks->scale = 0.0;
    }
}

__device__ void proj_solve_dev(const KState* pls, const double2* cvec, double2* d, double2* u, double2* g,
                               double2* ds) {
    const int lane = threadIdx.x & 31;
    const int k = pls->j;
    for (int i = lane; i < KLD; i += 32) g[i] = (i <= k) ? cvec[i] : z0();
    __syncwarp();
    if (lane == 0)
        for (int t = 0; t < pls->nrot; ++t) rot_apply(pls->rc[t], pls->rs[t], g[pls->ra[t]], g[pls->rb[t]]);
    __syncwarp();
    solve_upper(pls->R, g, ds, k, nullptr);
    __syncwarp();
    for (int i = lane; i < k; i += 32) d[i] = ds[i];
    for (int i = lane; i <= k; i += 32) {
        double2 acc = z0();
        for (int l = 0; l < k; ++l) acc = cfma(pls->H[i + KLD * l], ds[l], acc);
        u[i] = acc;
    }
}
__global__ void k_proj_solve(const KState* pls, const double2* cvec, double2* d, double2* u) {
    __shared__ double2 g[KLD];
    __shared__ double2 ds[KMAX];
    proj_solve_dev(pls, cvec, d, u, g, ds);
}
__global__ void k_bproj_solve(const KState* pls, const double2* cvec, long cs, double2* d, long dst, double2* u,
                              long us, Gate act) {
    __shared__ double2 g[KLD];
    __shared__ double2 ds[KMAX];
    const int r = blockIdx.x;
    if (!gate_open(act, r)) return;
    proj_solve_dev(pls, cvec + r * cs, d + r * dst, u + r * us, g, ds);
}

__global__ void k_set(double* out, double v) {
    if (threadIdx.x == 0) *out = v;
}

__global__ void k_cg_init(const double* r2, double* rr, double* nb2, double tol, int* active, int* iters) {
    if (threadIdx.x != 0) return;
    const double v = *r2;
    *rr = v;
    *nb2 = v;
    *iters = 0;
    *active = (v > 0.0 && v > tol * tol * v) ? 1 : 0;
}

__global__ void k_cg_scalars(double* rr, const double* rr_new, const double* nb2, double tol, int* active,
                             int* iters) {
    if (threadIdx.x != 0 || *active != 1) return;
    *rr = *rr_new;
    *iters += 1;
    *active = (*rr_new > tol * tol * *nb2) ? 1 : 0;
}

__global__ void k_rsqrt(double* out, const double* in) {
    if (threadIdx.x == 0) {
        const double v = *in;
        *out = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    }
}

// ------------------------------------------------------------ DR restart ----
constexpr int DR_THREADS = 128;
constexpr int LDS = KMAX;  // leading dimension of the shared matrices

struct DRSmem {
    double2 T[LDS * LDS];  // eigenproblem matrix -> Schur form
    double2 Q[LDS * LDS];  // accumulated unitary
    double2 G[KLD * (KMAX + 1)];  // harmonic Ritz vectors -> P (leading dimension KLD)
    double2 v[KLD];
    double2 f[KLD];
    double2 rot_s[KLD];
    double rot_c[KLD];
    double red[DR_THREADS];
    double2 redz[DR_THREADS];
    int sel[KMAX];
    int ctl[4];
    double2 mu;
};

__device__ double2 block_dot(const double2* a, const double2* b, int n, DRSmem& S) {
    // sum_i conj(a_i) b_i (n <= KLD), returned to every thread: each warp
    // computes it alone with a butterfly, so every lane of every warp holds the
    // same value and no block barrier is needed
    (void)S;
    const int lane = threadIdx.x & 31;
    double2 acc = z0();
    for (int i = lane; i < n; i += 32) acc = cfmac(a[i], b[i], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    return acc;
}

__global__ void __launch_bounds__(DR_THREADS) k_dr_restart(const KState* __restrict__ ks, DRState* dr, int k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DRSmem& S = *reinterpret_cast<DRSmem*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = ks->j;
    const double eps = 2.220446049250313e-16;
    if (tid == 0) dr->err = 0;

    // (a) T = H_n, Q = H_n^H (elimination workspace), f = e_n
    for (int e = tid; e < n * n; e += nt) {
        const int i = e % n, c = e / n;
        S.T[i + LDS * c] = ks->H[i + KLD * c];
        S.Q[i + LDS * c] = conj_(ks->H[c + KLD * i]);
    }
    for (int i = tid; i < n; i += nt) S.f[i] = (i == n - 1) ? make_double2(1.0, 0.0) : z0();
    __syncthreads();
    // (b) solve H_n^H f = e_n by Gaussian elimination with partial pivoting
    for (int p = 0; p < n; ++p) {
        if (tid == 0) {
            int best = p;
            double bv = cabs2d(S.Q[p + LDS * p]);
            for (int r = p + 1; r < n; ++r) {
                const double v = cabs2d(S.Q[r + LDS * p]);
                if (v > bv) { bv = v; best = r; }
            }
            S.ctl[0] = best;
            if (bv == 0.0) dr->err = 3;
        }
        __syncthreads();
        const int best = S.ctl[0];
        if (best != p) {
            for (int c = tid; c < n; c += nt) {
                const double2 t = S.Q[p + LDS * c];
                S.Q[p + LDS * c] = S.Q[best + LDS * c];
                S.Q[best + LDS * c] = t;
            }
            if (tid == 0) {
                const double2 t = S.f[p];
                S.f[p] = S.f[best];
                S.f[best] = t;
            }
        }
        __syncthreads();
        const double2 piv = S.Q[p + LDS * p];
        for (int r = p + 1 + tid; r < n; r += nt) {
            const double2 fac = (piv.x == 0.0 && piv.y == 0.0) ? z0() : cdiv(S.Q[r + LDS * p], piv);
            for (int c = p; c < n; ++c) S.Q[r + LDS * c] = csub(S.Q[r + LDS * c], cmul(fac, S.Q[p + LDS * c]));
            S.f[r] = csub(S.f[r], cmul(fac, S.f[p]));
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int i = n - 1; i >= 0; --i) {
            double2 acc = S.f[i];
            for (int c = i + 1; c < n; ++c) acc = csub(acc, cmul(S.Q[i + LDS * c], S.f[c]));
            const double2 piv = S.Q[i + LDS * i];
            S.f[i] = (piv.x == 0.0 && piv.y == 0.0) ? z0() : cdiv(acc, piv);
        }
    }
    __syncthreads();
    // (c) T[:, n-1] += |h_{n+1,n}|^2 f
    {
        const double h2 = cabs2(ks->H[n + KLD * (n - 1)]);
        for (int i = tid; i < n; i += nt) S.T[i + LDS * (n - 1)] = cadd(S.T[i + LDS * (n - 1)], cscale(S.f[i], h2));
    }
    // Q = I
    for (int e = tid; e < n * n; e += nt) {
        const int i = e % n, c = e / n;
        S.Q[i + LDS * c] = (i == c) ? make_double2(1.0, 0.0) : z0();
    }
    __syncthreads();
    // (d) Householder reduction to upper Hessenberg form, Q accumulated
    for (int p = 0; p + 2 < n; ++p) {
        // v = x + e^{i arg x0} ||x|| e1 over rows p+1..n-1
        if (tid == 0) {
            double a2 = 0.0;
            for (int r = p + 1; r < n; ++r) a2 += cabs2(S.T[r + LDS * p]);
            const double alpha = sqrt(a2);
            const double2 x0 = S.T[(p + 1) + LDS * p];
            const double ax0 = cabsd(x0);
            const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
            double vn2 = 0.0;
            for (int r = p + 1; r < n; ++r) {
                double2 vr = S.T[r + LDS * p];
                if (r == p + 1) vr = cadd(vr, cscale(ph, alpha));
                S.v[r] = vr;
                vn2 += cabs2(vr);
            }
            S.red[0] = (alpha == 0.0 || vn2 == 0.0) ? 0.0 : 2.0 / vn2;
        }
        __syncthreads();
        const double tau = S.red[0];
        if (tau != 0.0) {
            // left: rows p+1..n-1, columns p..n-1
            for (int c = p + tid; c < n; c += nt) {
                double2 s = z0();
                for (int r = p + 1; r < n; ++r) s = cfmac(S.v[r], S.T[r + LDS * c], s);
                s = cscale(s, tau);
                for (int r = p + 1; r < n; ++r) S.T[r + LDS * c] = csub(S.T[r + LDS * c], cmul(S.v[r], s));
            }
            __syncthreads();
            // right: all rows, columns p+1..n-1; and Q
            for (int r = tid; r < 2 * n; r += nt) {
                double2* M = (r < n) ? S.T : S.Q;
                const int rr = (r < n) ? r : r - n;
                double2 s = z0();
                for (int c = p + 1; c < n; ++c) s = cfma(M[rr + LDS * c], S.v[c], s);
                s = cscale(s, tau);
                for (int c = p + 1; c < n; ++c) M[rr + LDS * c] = csub(M[rr + LDS * c], cmul(s, conj_(S.v[c])));
            }
            __syncthreads();
        }
        for (int r = p + 2 + tid; r < n; r += nt) S.T[r + LDS * p] = z0();
        __syncthreads();
    }
    // (e) shifted complex QR iterations to the Schur form T = Q^+ T0 Q
    if (tid == 0) {
        S.ctl[1] = n - 1;  // hi
        S.ctl[2] = 0;      // iterations on the current eigenvalue
        S.ctl[3] = 0;      // total iterations
    }
    __syncthreads();
    while (true) {
        if (tid == 0) {
            int hi = S.ctl[1];
            int l = -1;
            while (hi > 0) {
                l = hi;
                while (l > 0) {
                    // magnitudes |re| + |im| (within a factor sqrt(2) of the modulus)
                    const double sub = cabs1d(S.T[l + LDS * (l - 1)]);
                    const double dsum = cabs1d(S.T[(l - 1) + LDS * (l - 1)]) + cabs1d(S.T[l + LDS * l]);
                    if (sub <= eps * dsum || sub < 1e-300) break;
                    --l;
                }
                if (l == hi) {  // deflate one eigenvalue
                    S.T[hi + LDS * (hi - 1)] = z0();
                    --hi;
                    S.ctl[2] = 0;
                    continue;
                }
                break;
            }
            S.ctl[1] = hi;
            S.ctl[0] = l;
            if (hi > 0) {
                if (l > 0) S.T[l + LDS * (l - 1)] = z0();
                const double2 a = S.T[(hi - 1) + LDS * (hi - 1)], b = S.T[(hi - 1) + LDS * hi];
                const double2 c = S.T[hi + LDS * (hi - 1)], d = S.T[hi + LDS * hi];
                double2 mu;
                if (S.ctl[2] > 0 && S.ctl[2] % 10 == 0) {
                    mu = cadd(d, make_double2(0.75 * cabsd(c), 0.0));  // exceptional shift
                } else {
                    const double2 hdiff = cscale(csub(a, d), 0.5);
                    const double2 disc2 = cadd(cmul(hdiff, hdiff), cmul(b, c));
                    // principal complex square root
                    const double m = cabsd(disc2);
                    double2 sq = make_double2(sqrt(0.5 * (m + disc2.x)), 0.0);
                    sq.y = (disc2.y >= 0.0 ? 1.0 : -1.0) * sqrt(fmax(0.5 * (m - disc2.x), 0.0));
                    const double2 mid = cscale(cadd(a, d), 0.5);
                    const double2 m1 = cadd(mid, sq), m2 = csub(mid, sq);
                    mu = (cabs2d(csub(m1, d)) <= cabs2d(csub(m2, d))) ? m1 : m2;
                }
                S.mu = mu;
                S.ctl[2] += 1;
                S.ctl[3] += 1;
                if (S.ctl[3] > 60 * n) {
                    dr->err = 4;
                    S.ctl[1] = 0;
                }
            }
        }
        __syncthreads();
        const int hi = S.ctl[1], l = S.ctl[0];
        if (hi <= 0) break;
        const double2 mu = S.mu;
        for (int i = l + tid; i <= hi; i += nt) S.T[i + LDS * i] = csub(S.T[i + LDS * i], mu);
        __syncthreads();
        for (int i = l; i < hi; ++i) {
            if (tid == 0) {
                double c;
                double2 s, r;
                givens(S.T[i + LDS * i], S.T[(i + 1) + LDS * i], c, s, r);
                S.rot_c[i] = c;
                S.rot_s[i] = s;
            }
            __syncthreads();
            const double c = S.rot_c[i];
            const double2 s = S.rot_s[i];
            for (int col = i + tid; col < n; col += nt) rot_apply(c, s, S.T[i + LDS * col], S.T[(i + 1) + LDS * col]);
            __syncthreads();
        }
        for (int i = l; i < hi; ++i) {
            const double c = S.rot_c[i];
            const double2 s = S.rot_s[i];
            const int rmax = min(i + 2, hi);
            // columns (i, i+1) times G^+: col_i' = c col_i + conj(s) col_{i+1}, col_{i+1}' = -s col_i + c col_{i+1}
            for (int r = tid; r < n + rmax + 1; r += nt) {
                double2* M = (r <= rmax) ? S.T : S.Q;
                const int rr = (r <= rmax) ? r : r - rmax - 1;
                const double2 a = M[rr + LDS * i], b = M[rr + LDS * (i + 1)];
                M[rr + LDS * i] = cadd(cscale(a, c), cmul(conj_(s), b));
                M[rr + LDS * (i + 1)] = csub(cscale(b, c), cmul(s, a));
            }
            __syncthreads();
        }
        for (int i = l + tid; i <= hi; i += nt) S.T[i + LDS * i] = cadd(S.T[i + LDS * i], mu);
        __syncthreads();
    }
    // (f) select the k eigenvalues of smallest modulus (stable in the index)
    if (tid == 0) {
        int idx[KMAX];
        for (int i = 0; i < n; ++i) idx[i] = i;
        for (int i = 1; i < n; ++i) {  // insertion sort: stable
            const int t = idx[i];
            const double vt = cabs2d(S.T[t + LDS * t]);
            int q = i - 1;
            while (q >= 0 && cabs2d(S.T[idx[q] + LDS * idx[q]]) > vt) {
                idx[q + 1] = idx[q];
                --q;
            }
            idx[q + 1] = t;
        }
        for (int i = 0; i < k; ++i) {
            S.sel[i] = idx[i];
            dr->theta[i] = S.T[idx[i] + LDS * idx[i]];
        }
    }
    __syncthreads();
    // (g) eigenvectors: back substitution in T, then g = Q y (column a of G)
    {
        // max |T_ij|, shared out over the CTA: strided maxima of |T_ij|^2, a warp
        // butterfly, then the warps' maxima
        double t2 = 0.0;
        for (int e = tid; e < n * n; e += nt) t2 = fmax(t2, cabs2d(S.T[(e % n) + LDS * (e / n)]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t2 = fmax(t2, __shfl_xor_sync(0xffffffffu, t2, o));
        if ((tid & 31) == 0) S.red[tid >> 5] = t2;
        __syncthreads();
        double tmax2 = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) tmax2 = fmax(tmax2, S.red[w]);
        const double small = fmax(eps * sqrt(tmax2), 1e-300);
        for (int a = tid; a < k; a += nt) {
            const int q = S.sel[a];
            const double2 th = S.T[q + LDS * q];
            double2 y[KMAX];
            for (int r = 0; r < n; ++r) y[r] = z0();
            y[q] = make_double2(1.0, 0.0);
            for (int r = q - 1; r >= 0; --r) {
                double2 s = z0();
                for (int m = r + 1; m <= q; ++m) s = cfma(S.T[r + LDS * m], y[m], s);
                double2 den = csub(S.T[r + LDS * r], th);
                const double dd = cabs2d(den);
                if (dd < small * small || dd == 0.0) den = make_double2(small, 0.0);
                y[r] = cneg(cdiv(s, den));
            }
            for (int r = 0; r < n; ++r) {
                double2 s = z0();
                for (int m = 0; m <= q; ++m) s = cfma(S.Q[r + LDS * m], y[m], s);
                S.G[r + KLD * a] = s;
            }
            S.G[n + KLD * a] = z0();
        }
    }
    __syncthreads();
    // (h) orthonormalise the k vectors (Gram-Schmidt, twice) -> P[:, :k]
    for (int a = 0; a < k; ++a) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int b = 0; b < a; ++b) {
                const double2 dt = block_dot(S.G + KLD * b, S.G + KLD * a, n, S);
                for (int r = tid; r < n; r += nt) S.G[r + KLD * a] = csub(S.G[r + KLD * a], cmul(dt, S.G[r + KLD * b]));
                __syncthreads();
            }
        }
        const double2 nn = block_dot(S.G + KLD * a, S.G + KLD * a, n, S);
        const double inv = nn.x > 0.0 ? 1.0 / sqrt(nn.x) : 0.0;
        if (nn.x <= 0.0 && tid == 0) dr->err = 5;
        for (int r = tid; r < n; r += nt) S.G[r + KLD * a] = cscale(S.G[r + KLD * a], inv);
        __syncthreads();
    }
    // (i) last column: rho orthonormalised against the first k (twice); length n+1
    for (int r = tid; r <= n; r += nt) S.G[r + KLD * k] = ks->rho[r];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int b = 0; b < k; ++b) {
            const double2 dt = block_dot(S.G + KLD * b, S.G + KLD * k, n + 1, S);
            for (int r = tid; r <= n; r += nt) S.G[r + KLD * k] = csub(S.G[r + KLD * k], cmul(dt, S.G[r + KLD * b]));
            __syncthreads();
        }
    }
    {
        const double2 nn = block_dot(S.G + KLD * k, S.G + KLD * k, n + 1, S);
        const double inv = nn.x > 0.0 ? 1.0 / sqrt(nn.x) : 0.0;
        if (nn.x <= 0.0 && tid == 0) dr->err = 6;
        for (int r = tid; r <= n; r += nt) S.G[r + KLD * k] = cscale(S.G[r + KLD * k], inv);
    }
    __syncthreads();
    for (int e = tid; e < (n + 1) * (k + 1); e += nt) {
        const int r = e % (n + 1), a = e / (n + 1);
        dr->P[r + KLD * a] = S.G[r + KLD * a];
    }
    __syncthreads();
    // (j) Y = H P_k  -> T (rows n+1, cols k), then H_k = P^+ Y ; (k) c = P^+ rho
    for (int e = tid; e < (n + 1) * k; e += nt) {
        const int r = e % (n + 1), a = e / (n + 1);
        double2 s = z0();
        for (int m = 0; m < n; ++m) s = cfma(ks->H[r + KLD * m], dr->P[m + KLD * a], s);
        S.Q[r + (n + 1) * a] = s;  // Q is free now; ld n+1
    }
    __syncthreads();
    for (int e = tid; e < (k + 1) * k; e += nt) {
        const int r = e % (k + 1), a = e / (k + 1);
        double2 s = z0();
        for (int m = 0; m <= n; ++m) s = cfmac(dr->P[m + KLD * r], S.Q[m + (n + 1) * a], s);
        dr->Hk[r + KLD * a] = s;
    }
    for (int r = tid; r <= k; r += nt) {
        double2 s = z0();
        for (int m = 0; m <= n; ++m) s = cfmac(dr->P[m + KLD * r], ks->rho[m], s);
        dr->ck[r] = s;
    }
    if (tid == 0) {
        dr->j = n;
        dr->k = k;
    }
}

}  // namespace

void ks_start(KState* ks, const double* nrm2, double tol_rel, const double* nb2, cudaStream_t s) {
    k_ks_start<<<1, 32, 0, s>>>(ks, nrm2, tol_rel, nb2);
    count_launch();
}
void bks_start(KState* ks, int nb, const double* nrm2, long ns, double tol_rel, const double* nb2, long nbs, Gate act,
               cudaStream_t s) {
    k_bks_start<<<nb, 32, 0, s>>>(ks, nrm2, ns, tol_rel, nb2, nbs, act);
    count_launch();
}
void bks_push(KState* ks, int nb, int jh, cudaStream_t s) {
    k_bks_push<<<nb, 32, 0, s>>>(ks, jh);
    count_launch();
}
void bks_finish(KState* ks, int nb, cudaStream_t s) {
    k_bks_finish<<<nb, 32, 0, s>>>(ks);
    count_launch();
}
void bproj_solve(const KState* pls, int nb, const double2* cvec, long cs, double2* d, long ds, double2* u, long us,
                 Gate act, cudaStream_t s) {
    k_bproj_solve<<<nb, 32, 0, s>>>(pls, cvec, cs, d, ds, u, us, act);
    count_launch();
}
void scalar_set(double* out, double v, cudaStream_t s) {
    k_set<<<1, 32, 0, s>>>(out, v);
    count_launch();
}
void cg_init(const double* r2, double* rr, double* nb2, double tol, int* active, int* iters, cudaStream_t s) {
    k_cg_init<<<1, 32, 0, s>>>(r2, rr, nb2, tol, active, iters);
    count_launch();
}
void cg_scalars(double* rr, const double* rr_new, const double* nb2, double tol, int* active, int* iters,
                cudaStream_t s) {
    k_cg_scalars<<<1, 32, 0, s>>>(rr, rr_new, nb2, tol, active, iters);
    count_launch();
}
void ks_push(KState* ks, int jh, cudaStream_t s) {
    k_ks_push<<<1, 32, 0, s>>>(ks, jh);
    count_launch();
}
void ks_finish(KState* ks, cudaStream_t s) {
    k_ks_finish<<<1, 32, 0, s>>>(ks);
    count_launch();
}
void ks_load_dense(KState* ks, const double2* Hk, const double2* ck, int k, double tol_abs, cudaStream_t s) {
    k_ks_load_dense<<<1, 32, 0, s>>>(ks, Hk, ck, k, tol_abs);
    count_launch();
}
void proj_solve(const KState* pls, const double2* cvec, double2* d, double2* u, cudaStream_t s) {
    k_proj_solve<<<1, 32, 0, s>>>(pls, cvec, d, u);
    count_launch();
}
void scalar_rsqrt(double* out, const double* in, cudaStream_t s) {
    k_rsqrt<<<1, 32, 0, s>>>(out, in);
    count_launch();
}

mg_status dr_restart(const KState* ks, DRState* dr, int k, cudaStream_t s) {
    static int configured = -1;
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (configured != dev) {
        MG_CUDA_TRY(cudaFuncSetAttribute(k_dr_restart, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(DRSmem)));
        configured = dev;
    }
    k_dr_restart<<<1, DR_THREADS, sizeof(DRSmem), s>>>(ks, dr, k);
    count_launch();
    MG_LAUNCH_CHECK();
    return MG_OK;
}

}  // namespace mg
