// The whole GMRES-Proj(m,k) coarsest-grid solve (Section 2; Morgan & Wilcox)
// in one cooperative persistent kernel.
//
// The coarsest grid is small (256 sites x 24 dofs at 256^2) and its solve runs
// ~10^3 Krylov steps per outer iteration, so a step is bound by latency, not by
// bytes: one launch per solve, three grid barriers per Arnoldi step, and the
// small least-squares work done redundantly (and identically) by every CTA.
//
// Work split: CTA b owns sites [b*spc, (b+1)*spc) and their 24 dofs; every
// vector operation touches only the CTA's own rows, except the stencil apply,
// which reads neighbour rows written by other CTAs before the previous barrier.
// Reductions: each CTA writes one partial per quantity, and after the barrier
// every CTA sums all partials in CTA order with the same warp tree, so every
// CTA holds bit-identical scalars and takes identical control decisions.
//
// Per Arnoldi step j (CGS2, as in the rest of the library):
//   [sync] w = A v_j; h1 = V^+ w (partials)
//   [sync] reduce h1; w -= V h1; h2 = V^+ w, n2 = ||w||^2 (partials)
//   [sync] reduce h2, n2; w -= V h2; ||w||^2 = n2 - |h2|^2 (V orthonormal);
//          Givens update of the least squares; v_{j+1} = w / h_{j+1,j}
#include <cooperative_groups.h>

#include "coarse_coop.cuh"

namespace cg = cooperative_groups;

namespace mg {

namespace {

constexpr int CO_THREADS = 256;
constexpr int CO_WARPS = CO_THREADS / 32;
constexpr int NDOF = 24;

struct CoopSmem {
    double2 H[(MSMAX + 1) * MSMAX];  // column-major, ld MSMAX + 1
    double2 R[(MSMAX + 1) * MSMAX];
    double rc[MSMAX];
    double2 rs[MSMAX];
    double2 g[MSMAX + 1], c[MSMAX + 1], d[MSMAX], rho[MSMAX + 1];
    double2 red[PSTR];               // reduced quantities of the current phase
    double2 h1[MSMAX + 1];
    double2 pd[KMAX], pu[KLD];       // projection coefficients
    double scal[8];
    int ctl[8];
};

__device__ __forceinline__ double cabsd(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
    const double ab = cabsd(b);
    if (ab == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); r = a; return; }
    const double aa = cabsd(a);
    if (aa == 0.0) { c = 0.0; s = make_double2(b.x / ab, -b.y / ab); r = make_double2(ab, 0.0); return; }
    const double rh = hypot(aa, ab);
    c = aa / rh;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    s = cscale(cmul(ph, conj_(b)), 1.0 / rh);
    r = cscale(ph, rh);
}
__device__ __forceinline__ void rot_apply(double c, double2 s, double2& up, double2& uq) {
    const double2 p = up, q = uq;
    up = cadd(cscale(p, c), cmul(s, q));
    uq = csub(cscale(q, c), cmul(conj_(s), p));
}

// Partials of nd inner products conj(X[i]) . y over the CTA's rows (warp per
// product, lanes over rows), plus optionally ||y||^2 in slot nd.  Written to
// part[blockIdx.x * PSTR + i].
template <typename T>
__device__ void partial_gram(const C2<T>* X, long ldx, int nd, const C2<T>* y, long r0, int nrows, bool norm,
                             double2* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntot = nd + (norm ? 1 : 0);
    for (int i = warp; i < ntot; i += CO_WARPS) {
        C2<T> acc = mk<T>(0, 0);
        if (i < nd) {
            const C2<T>* xi = X + (long)i * ldx + r0;
            for (int e = lane; e < nrows; e += 32) acc = cfmac(xi[e], y[r0 + e], acc);
        } else {
            for (int e = lane; e < nrows; e += 32) {
                const C2<T> v = y[r0 + e];
                acc.x += v.x * v.x + v.y * v.y;
            }
        }
        double2 a = to_d2(acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        }
        if (lane == 0) part[(size_t)blockIdx.x * PSTR + i] = a;
    }
}

// Sum the partials of all CTAs in CTA order (every CTA computes the same
// result): red[i] = sum_b part[b * PSTR + i], i < n.
__device__ void reduce_partials(const double2* part, int n, double2* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    for (int i = warp; i < n; i += CO_WARPS) {
        double2 a = make_double2(0.0, 0.0);
        for (int b = lane; b < G; b += 32) a = cadd(a, __ldcg(part + (size_t)b * PSTR + i));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        }
        if (lane == 0) red[i] = a;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(CO_THREADS) k_coarse_proj(CoopArgs<T> a) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CoopSmem& S = *reinterpret_cast<CoopSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const long nsite = (long)a.Nx * a.Nt;
    const long n = nsite * NDOF;
    const long s0 = (long)blockIdx.x * a.spc;
    const long s1 = min(nsite, s0 + a.spc);
    const long r0 = s0 * NDOF;
    const int nrows = (int)max(0L, (s1 - s0) * NDOF);
    const int k = a.k, ms = a.ms;
    double2* partA = a.part;
    double2* partB = a.part + (size_t)gridDim.x * PSTR;

    // x = 0, r = f, ||f||^2
    for (int e = tid; e < nrows; e += CO_THREADS) {
        a.x[r0 + e] = mk<T>(0, 0);
        a.r[r0 + e] = a.f[r0 + e];
    }
    __syncthreads();
    partial_gram<T>(a.r, 0, 0, a.r, r0, nrows, true, partA);
    grid.sync();
    reduce_partials(partA, 1, S.red);
    const double nb = sqrt(fmax(S.red[0].x, 0.0));
    const double tol_abs = a.tol * nb;
    int iters = 0, cycles = 0, conv = 0;
    while (true) {
        // ---- projection onto the deflation space: d = argmin ||W^+ r - H_k d|| ----
        partial_gram<T>(a.W, n, k + 1, a.r, r0, nrows, false, partB);
        grid.sync();
        reduce_partials(partB, k + 1, S.red);
        if (tid == 0) {
            const KState* P = a.pls;
            double2 g[KLD];
            for (int i = 0; i <= k; ++i) g[i] = S.red[i];
            for (int t = 0; t < P->nrot; ++t) rot_apply(P->rc[t], P->rs[t], g[P->ra[t]], g[P->rb[t]]);
            for (int i = k - 1; i >= 0; --i) {
                double2 acc = g[i];
                for (int l = i + 1; l < k; ++l) acc = csub(acc, cmul(P->R[i + KLD * l], S.pd[l]));
                S.pd[i] = cdiv(acc, P->R[i + KLD * i]);
            }
            for (int i = 0; i <= k; ++i) {
                double2 acc = make_double2(0.0, 0.0);
                for (int l = 0; l < k; ++l) acc = cfma(P->H[i + KLD * l], S.pd[l], acc);
                S.pu[i] = acc;
            }
        }
        __syncthreads();
        for (int e = tid; e < nrows; e += CO_THREADS) {
            C2<T> xv = a.x[r0 + e], rv = a.r[r0 + e];
            for (int i = 0; i < k; ++i) xv = cfma(a.W[(long)i * n + r0 + e], from_d2<T>(S.pd[i]), xv);
            for (int i = 0; i <= k; ++i) rv = csub(rv, cmul(a.W[(long)i * n + r0 + e], from_d2<T>(S.pu[i])));
            a.x[r0 + e] = xv;
            a.r[r0 + e] = rv;
        }
        __syncthreads();
        partial_gram<T>(a.r, 0, 0, a.r, r0, nrows, true, partA);
        grid.sync();
        reduce_partials(partA, 1, S.red);
        const double beta = sqrt(fmax(S.red[0].x, 0.0));
        if (beta <= tol_abs || beta == 0.0) {
            conv = 1;
            break;
        }
        // ---- one GMRES(ms) cycle from r ----
        // (shared memory is not zero-initialised: H must be zero below its subdiagonal)
        for (int e = tid; e < (MSMAX + 1) * MSMAX; e += CO_THREADS) {
            S.H[e] = make_double2(0.0, 0.0);
            S.R[e] = make_double2(0.0, 0.0);
        }
        if (tid == 0) {
            for (int i = 0; i <= ms; ++i) {
                S.c[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
                S.g[i] = S.c[i];
            }
            S.scal[0] = 1.0 / beta;
        }
        __syncthreads();
        {
            const T sc = (T)S.scal[0];
            for (int e = tid; e < nrows; e += CO_THREADS) a.V[r0 + e] = cscale(a.r[r0 + e], sc);
        }
        int j = 0, stop = 0;
        for (; j < ms && !stop; ++j) {
            grid.sync();  // v_j complete everywhere
            C2<T>* vj = a.V + (long)j * n;
            C2<T>* w = a.V + (long)(j + 1) * n;
            // w = A v_j on the CTA's rows (column-major 24x24 blocks)
            for (int e = tid; e < nrows; e += CO_THREADS) {
                const long s = s0 + e / NDOF;
                const int kk = e % NDOF;
                const int xx = (int)(s % a.Nx), tt = (int)(s / a.Nx);
                const long nb5[5] = {s, (xx + 1 == a.Nx) ? s - xx : s + 1, (xx == 0) ? s + a.Nx - 1 : s - 1,
                                     (tt + 1 == a.Nt) ? (long)xx : s + a.Nx,
                                     (tt == 0) ? s + (long)a.Nx * (a.Nt - 1) : s - a.Nx};
                const C2<T>* Ab = a.A + s * (5L * NDOF * NDOF) + kk;
                C2<T> acc = mk<T>(0, 0);
#pragma unroll
                for (int d = 0; d < 5; ++d) {
                    // neighbour rows were written by other CTAs: read through L2 (L1 is not coherent)
                    const C2<T>* xv = vj + nb5[d] * NDOF;
#pragma unroll 8
                    for (int l = 0; l < NDOF; ++l) acc = cfma(Ab[(d * NDOF + l) * NDOF], __ldcg(xv + l), acc);
                }
                w[r0 + e] = acc;
            }
            __syncthreads();
            partial_gram<T>(a.V, n, j + 1, w, r0, nrows, false, partB);
            grid.sync();
            reduce_partials(partB, j + 1, S.red);
            for (int i = tid; i <= j; i += CO_THREADS) S.h1[i] = S.red[i];
            __syncthreads();
            for (int e = tid; e < nrows; e += CO_THREADS) {
                C2<T> wv = w[r0 + e];
                for (int i = 0; i <= j; ++i) wv = csub(wv, cmul(a.V[(long)i * n + r0 + e], from_d2<T>(S.h1[i])));
                w[r0 + e] = wv;
            }
            __syncthreads();
            partial_gram<T>(a.V, n, j + 1, w, r0, nrows, true, partA);
            grid.sync();
            reduce_partials(partA, j + 2, S.red);
            if (tid == 0) {
                double h2n = 0.0;
                for (int i = 0; i <= j; ++i) {
                    const double2 hh = cadd(S.h1[i], S.red[i]);
                    S.H[i + (MSMAX + 1) * j] = hh;
                    S.R[i + (MSMAX + 1) * j] = hh;
                    h2n += cabs2(S.red[i]);
                }
                const double hn = sqrt(fmax(S.red[j + 1].x - h2n, 0.0));
                S.H[(j + 1) + (MSMAX + 1) * j] = make_double2(hn, 0.0);
                S.R[(j + 1) + (MSMAX + 1) * j] = make_double2(hn, 0.0);
                double2* Rc = S.R + (MSMAX + 1) * j;
                for (int t = 0; t < j; ++t) rot_apply(S.rc[t], S.rs[t], Rc[t], Rc[t + 1]);
                double cc;
                double2 ss, rr;
                givens(Rc[j], Rc[j + 1], cc, ss, rr);
                Rc[j] = rr;
                Rc[j + 1] = make_double2(0.0, 0.0);
                S.rc[j] = cc;
                S.rs[j] = ss;
                rot_apply(cc, ss, S.g[j], S.g[j + 1]);
                const double res = cabsd(S.g[j + 1]);
                S.ctl[0] = (res <= tol_abs) ? 1 : 0;
                S.ctl[1] = (hn == 0.0) ? 1 : 0;
                S.scal[1] = hn > 0.0 ? 1.0 / hn : 0.0;
            }
            __syncthreads();
            {
                const T sc = (T)S.scal[1];
                for (int e = tid; e < nrows; e += CO_THREADS) {
                    C2<T> wv = w[r0 + e];
                    for (int i = 0; i <= j; ++i)
                        wv = csub(wv, cmul(a.V[(long)i * n + r0 + e], from_d2<T>(S.red[i])));
                    w[r0 + e] = cscale(wv, sc);
                }
            }
            ++iters;
            conv = S.ctl[0];
            stop = S.ctl[0] | S.ctl[1];
            __syncthreads();
        }
        // ---- finish the cycle: d = R^{-1} g, rho = c - H d, x += V d, r = V rho ----
        const int jj = j;
        if (tid == 0) {
            for (int i = jj - 1; i >= 0; --i) {
                double2 acc = S.g[i];
                for (int l = i + 1; l < jj; ++l) acc = csub(acc, cmul(S.R[i + (MSMAX + 1) * l], S.d[l]));
                const double2 piv = S.R[i + (MSMAX + 1) * i];
                S.d[i] = (piv.x == 0.0 && piv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(acc, piv);
            }
            for (int i = 0; i <= jj; ++i) {
                double2 acc = S.c[i];
                for (int l = 0; l < jj; ++l) acc = csub(acc, cmul(S.H[i + (MSMAX + 1) * l], S.d[l]));
                S.rho[i] = acc;
            }
        }
        __syncthreads();
        for (int e = tid; e < nrows; e += CO_THREADS) {
            C2<T> xv = a.x[r0 + e];
            C2<T> rv = mk<T>(0, 0);
            for (int i = 0; i < jj; ++i) xv = cfma(a.V[(long)i * n + r0 + e], from_d2<T>(S.d[i]), xv);
            for (int i = 0; i <= jj; ++i) rv = cfma(a.V[(long)i * n + r0 + e], from_d2<T>(S.rho[i]), rv);
            a.x[r0 + e] = xv;
            a.r[r0 + e] = rv;
        }
        ++cycles;
        __syncthreads();
        if (conv || cycles >= a.max_cycles) break;
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.out->iters += iters;
        a.out->cycles += cycles;
        a.out->solves += 1;
        a.out->unconverged += conv ? 0 : 1;
    }
}

template <typename T>
struct Geometry {
    int grid = 0, spc = 0;
};

template <typename T>
mg_status geometry(long nsite, Geometry<T>& g) {
    static int max_active[16] = {0};
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 16) dev = 0;
    if (max_active[dev] == 0) {
        MG_CUDA_TRY(cudaFuncSetAttribute(k_coarse_proj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(CoopSmem)));
        int per_sm = 0;
        MG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_proj<T>, CO_THREADS,
                                                                  sizeof(CoopSmem)));
        max_active[dev] = per_sm * sm_count();
        if (max_active[dev] < 1) {
            set_error("the coarse solve kernel cannot be resident");
            return MG_ECUDA;
        }
    }
    // about 8 sites (192 rows) per CTA, at most one CTA per SM
    long G = (nsite + 7) / 8;
    G = std::min<long>(G, std::min<long>(sm_count(), max_active[dev]));
    G = std::max<long>(G, 1);
    g.spc = (int)((nsite + G - 1) / G);
    g.grid = (int)((nsite + g.spc - 1) / g.spc);
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
    Geometry<T> g;
    MG_TRY(geometry<T>((long)a.Nx * a.Nt, g));
    if (g.grid > a.part_ctas) {
        set_error("coarse solve: %d CTAs exceed the partial-sum buffer (%d)", g.grid, a.part_ctas);
        return MG_EINVAL;
    }
    a.spc = g.spc;
    void* params[] = {&a};
    MG_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_coarse_proj<T>, dim3(g.grid), dim3(CO_THREADS), params,
                                            sizeof(CoopSmem), s));
    count_launch();
    return MG_OK;
}

template mg_status launch_coarse_proj<double>(const CoopArgs<double>&, cudaStream_t);
template mg_status launch_coarse_proj<float>(const CoopArgs<float>&, cudaStream_t);

}  // namespace mg
