// Hierarchy set-up kernels (Section 2, first paragraph):
//  * chiral doubling + local 4^2 blocking + local orthonormalisation of the
//    globally orthonormalised near-null vectors into the prolongator Q;
//  * the Galerkin product D^ = P^+ D P as a 5-point stencil of 24x24 blocks.
// Both run once per hierarchy (not in the solve).
#include "setup.cuh"

namespace mg {

namespace {

constexpr int NV = 12;
constexpr int BL = 4;
constexpr int BS = 16;
constexpr int LO_THREADS = 192;

__device__ double2 cta_dot(const double2* a, const double2* b, int n, double2* red) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cfmac(a[i], b[i], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < (int)blockDim.x; ++i) t = cadd(t, red[i]);
        red[0] = t;
    }
    __syncthreads();
    const double2 r = red[0];
    __syncthreads();
    return r;
}

// One CTA per (coarse site B, chirality c): the 16h x 12 matrix of the
// chirality-c part of the 12 vectors on the block's sites, modified
// Gram-Schmidt over the vectors in order.
__global__ void __launch_bounds__(LO_THREADS) k_local_orth(double2* __restrict__ Q, const double2* __restrict__ V,
                                                           long ldv, int NxF, int h, double rank_tol, int* err) {
    __shared__ double2 M[NV][BS * 12];
    __shared__ double2 red[LO_THREADS];
    const int B = blockIdx.x >> 1, c = blockIdx.x & 1;
    const int NxC = NxF / BL;
    const int bx = B % NxC, bt = B / NxC;
    const int len = BS * h;
    for (int e = threadIdx.x; e < NV * len; e += blockDim.x) {
        const int j = e / len, r = e - j * len;
        const int l = r / h, a = r - l * h;
        const long fs = (long)(bt * BL + l / BL) * NxF + bx * BL + (l % BL);
        M[j][r] = V[(long)j * ldv + fs * 2 * h + c * h + a];
    }
    __syncthreads();
    for (int j = 0; j < NV; ++j) {
        const double before = sqrt(cta_dot(M[j], M[j], len, red).x);
        for (int i = 0; i < j; ++i) {
            const double2 ov = cta_dot(M[i], M[j], len, red);
            for (int r = threadIdx.x; r < len; r += blockDim.x) M[j][r] = csub(M[j][r], cmul(ov, M[i][r]));
            __syncthreads();
        }
        const double nrm = sqrt(cta_dot(M[j], M[j], len, red).x);
        if (!(nrm > rank_tol * before)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
        }
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int r = threadIdx.x; r < len; r += blockDim.x) M[j][r] = cscale(M[j][r], inv);
        __syncthreads();
    }
    double2* q = Q + ((long)B * 2 * NV + c * NV) * len;
    for (int e = threadIdx.x; e < NV * len; e += blockDim.x) q[e] = M[e / len][e % len];
}

// Entry (a, b) of the finer operator's block A[s][d] (dof x dof).
struct FinerWilson {
    const double2* U;
    double diag;
    int Lx, Lt;
    __device__ double2 operator()(long s, int d, int a, int b) const {
        const int x = (int)(s % Lx), t = (int)(s / Lx);
        if (d == 0) return make_double2(a == b ? diag : 0.0, 0.0);
        double2 u;
        double2 m;  // the spin matrix (1 -/+ sigma_mu) entry (a, b)
        double sign = 1.0;
        if (d == 1) {  // -1/2 (1 - sigma_1) U_x(s)
            u = U[2 * s];
            m = make_double2(a == b ? 1.0 : -1.0, 0.0);
        } else if (d == 2) {  // -1/2 (1 + sigma_1) U_x(s - x)^*
            const long sm = (x == 0) ? s + Lx - 1 : s - 1;
            u = conj_(U[2 * sm]);
            m = make_double2(1.0, 0.0);
        } else if (d == 3) {  // -1/2 (1 - sigma_2) U_t(s), (1 - sigma_2) = [[1, i], [-i, 1]]
            u = U[2 * s + 1];
            if (t == Lt - 1) sign = -1.0;
            m = (a == b) ? make_double2(1.0, 0.0) : (a == 0 ? make_double2(0.0, 1.0) : make_double2(0.0, -1.0));
        } else {  // -1/2 (1 + sigma_2) U_t(s - t)^*, (1 + sigma_2) = [[1, -i], [i, 1]]
            const long sm = (t == 0) ? s + (long)Lx * (Lt - 1) : s - Lx;
            u = conj_(U[2 * sm + 1]);
            if (t == 0) sign = -1.0;
            m = (a == b) ? make_double2(1.0, 0.0) : (a == 0 ? make_double2(0.0, -1.0) : make_double2(0.0, 1.0));
        }
        return cscale(cmul(u, m), -0.5 * sign);
    }
};

struct FinerStencil {
    const double2* A;  // [s][d][b][a] column-major blocks, dof 24
    __device__ double2 operator()(long s, int d, int a, int b) const {
        return A[((s * 5 + d) * 24 + b) * 24 + a];
    }
};

// One CTA per coarse site B; thread (k, l2) owns output entry (k, l2) of all
// five directions.  For every finer site s of the block and every term d of
// the finer operator:  T1 = A_f[s,d] P_nbr(s,d)  (dof x 24), then
//   Ac[B, dest] += P_s^+ T1,
// dest = d when the hop leaves the block through its face, else self.
template <typename F>
__global__ void __launch_bounds__(576) k_galerkin(double2* __restrict__ Ac, F Af, const double2* __restrict__ Q,
                                                  int NxF, int NtF, int h) {
    __shared__ double2 T1[24 * 24];
    const int B = blockIdx.x;
    const int NxC = NxF / BL;
    const int bx = B % NxC, bt = B / NxC;
    const int k = threadIdx.x % 24, l2 = threadIdx.x / 24;
    const int dof = 2 * h;
    double2 acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = make_double2(0.0, 0.0);
    const int ck = k / NV, jk = k % NV;
    for (int l = 0; l < BS; ++l) {
        const int lx = l % BL, lt = l / BL;
        const int xf = bx * BL + lx, tf = bt * BL + lt;
        const long s = (long)tf * NxF + xf;
        for (int d = 0; d < 5; ++d) {
            int xn = xf, tn = tf, dest = 0;
            if (d == 1) { xn = (xf + 1) % NxF; dest = (lx == BL - 1) ? 1 : 0; }
            if (d == 2) { xn = (xf + NxF - 1) % NxF; dest = (lx == 0) ? 2 : 0; }
            if (d == 3) { tn = (tf + 1) % NtF; dest = (lt == BL - 1) ? 3 : 0; }
            if (d == 4) { tn = (tf + NtF - 1) % NtF; dest = (lt == 0) ? 4 : 0; }
            const long sn = (long)tn * NxF + xn;
            const int Bn = (tn / BL) * NxC + xn / BL;
            const int ln = (xn % BL) + BL * (tn % BL);
            // stage 1: T1[a][l2'] = sum_b' A_f[s,d][a][c' h + b'] Q[Bn][c'][j'][ln][b']
            for (int e = threadIdx.x; e < dof * 24; e += blockDim.x) {
                const int a = e % dof, lc = e / dof;
                const int cl = lc / NV, jl = lc % NV;
                const double2* qn = Q + (((long)Bn * 2 * NV + cl * NV + jl) * BS + ln) * h;
                double2 s1 = make_double2(0.0, 0.0);
                for (int bb = 0; bb < h; ++bb) s1 = cfma(Af(s, d, a, cl * h + bb), qn[bb], s1);
                T1[a + dof * lc] = s1;
            }
            __syncthreads();
            // stage 2: term = sum_a' conj(Q[B][ck][jk][l][a']) T1[ck h + a'][l2]
            const double2* qs = Q + (((long)B * 2 * NV + ck * NV + jk) * BS + l) * h;
            double2 term = make_double2(0.0, 0.0);
            for (int aa = 0; aa < h; ++aa) term = cfmac(qs[aa], T1[(ck * h + aa) + dof * l2], term);
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (q == dest) acc[q] = cadd(acc[q], term);
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) Ac[(((long)B * 5 + q) * 24 + l2) * 24 + k] = acc[q];
}

}  // namespace

void launch_local_orth(double2* Q, const double2* V, long ldv, int NxF, int NtF, int h, double rank_tol, int* err,
                       cudaStream_t s) {
    const int nc = (NxF / BL) * (NtF / BL);
    k_local_orth<<<2 * nc, LO_THREADS, 0, s>>>(Q, V, ldv, NxF, h, rank_tol, err);
    count_launch();
}

void launch_galerkin_wilson(double2* Ac, const double2* U, double m0, const double2* Q, int Lx, int Lt,
                            cudaStream_t s) {
    const int nc = (Lx / BL) * (Lt / BL);
    FinerWilson f{U, m0 + 2.0, Lx, Lt};
    k_galerkin<FinerWilson><<<nc, 576, 0, s>>>(Ac, f, Q, Lx, Lt, 1);
    count_launch();
}

void launch_galerkin_stencil(double2* Ac, const double2* A, const double2* Q, int NxF, int NtF, cudaStream_t s) {
    const int nc = (NxF / BL) * (NtF / BL);
    FinerStencil f{A};
    k_galerkin<FinerStencil><<<nc, 576, 0, s>>>(Ac, f, Q, NxF, NtF, 12);
    count_launch();
}

}  // namespace mg
