// The intermediate-grid operator D^ = P^+ D P (Section 2) with low-rank hop
// blocks.  A hop block A[s][d] (d = +x, -x, +t, -t) couples the 16 sites of
// one 4^2 block to the 16 of its neighbour through the 4 site pairs across
// their common edge; each pair contributes P(x)^+ [-(1 -+ sigma_mu)/2 U] P(y),
// and (1 -+ sigma_mu)/2 is a rank-1 spin projector, so A[s][d] has rank <= 4.
// It is stored as factors Q R (Q: 24 x 4, R: 4 x 24): 192 complex entries
// instead of 576, and applied as y += Q (R x), with the self block dense.
//
// The factors are computed at set-up from the dense Galerkin blocks by
// Gram-Schmidt with column pivoting (four steps, one warp per block, FP64), so
// the factored operator equals the dense one to rounding whatever the
// conventions of the fine operator; the largest relative reconstruction
// error over the blocks is reported, and the caller keeps the dense operator
// if it is not at rounding level.
#include <algorithm>
#include <type_traits>

#include "ops.cuh"

namespace mg {

namespace {

constexpr int N = 24;
constexpr int LR_BLOCK = 2 * LR_RANK * N;  // Q then R of one hop direction
constexpr int LR_SPB = 8;                  // sites per block of the apply

__device__ __forceinline__ double2 wsum2(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one warp per (site, direction): d = 0 copies the self block, d = 1..4
// factors the hop block; lane k < 24 holds row k
__global__ void k_factor_hops(double2* __restrict__ F, const double2* __restrict__ A, long nsite,
                              unsigned long long* maxerr) {
    const int lane = threadIdx.x & 31;
    const long task = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (task >= nsite * 5) return;
    const long s = task / 5;
    const int d = (int)(task - s * 5);
    const double2* Ab = A + (s * 5 + d) * (long)(N * N);  // column-major: (k, l) at l * N + k
    double2* Fs = F + s * (long)LR_SITE;
    const bool row = lane < N;
    if (d == 0) {
        for (int e = lane; e < N * N; e += 32) Fs[e] = Ab[e];
        return;
    }
    double2* Q = Fs + N * N + (d - 1) * LR_BLOCK;  // [i][k]
    double2* R = Q + LR_RANK * N;                  // [i][l]
    double2 a[N];
#pragma unroll
    for (int l = 0; l < N; ++l) a[l] = row ? Ab[l * N + lane] : make_double2(0.0, 0.0);
    double nrm[N], anorm2 = 0.0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
        nrm[l] = wsum(a[l].x * a[l].x + a[l].y * a[l].y);
        anorm2 += nrm[l];
    }
    double2 q[LR_RANK];
#pragma unroll
    for (int i = 0; i < LR_RANK; ++i) {
        int p = 0;
#pragma unroll
        for (int l = 1; l < N; ++l)
            if (nrm[l] > nrm[p]) p = l;
        double2 ap = a[0];
#pragma unroll
        for (int l = 1; l < N; ++l)
            if (l == p) ap = a[l];
        const bool keep = nrm[p] > 1e-28 * anorm2;
        const double inv = keep ? rsqrt(nrm[p]) : 0.0;
        q[i] = make_double2(ap.x * inv, ap.y * inv);
        // a second pass against the earlier directions keeps Q orthonormal to
        // rounding, so Q Q^+ is the projector the reconstruction relies on
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const double2 c = wsum2(make_double2(q[j].x * q[i].x + q[j].y * q[i].y, q[j].x * q[i].y - q[j].y * q[i].x));
            q[i].x -= q[j].x * c.x - q[j].y * c.y;
            q[i].y -= q[j].x * c.y + q[j].y * c.x;
        }
        if (keep) {
            const double qn = wsum(q[i].x * q[i].x + q[i].y * q[i].y);
            const double qi = qn > 0.0 ? rsqrt(qn) : 0.0;
            q[i] = make_double2(q[i].x * qi, q[i].y * qi);
        }
        // remove q_i from every column, and the next pivot norms from the updated columns
#pragma unroll
        for (int l = 0; l < N; ++l) {
            const double2 c = wsum2(make_double2(q[i].x * a[l].x + q[i].y * a[l].y, q[i].x * a[l].y - q[i].y * a[l].x));
            a[l].x -= q[i].x * c.x - q[i].y * c.y;
            a[l].y -= q[i].x * c.y + q[i].y * c.x;
            nrm[l] = wsum(a[l].x * a[l].x + a[l].y * a[l].y);
        }
        if (row) Q[i * N + lane] = q[i];
    }
    // R = Q^+ A (the original block), and the reconstruction error
    double err2 = 0.0;
    double2 rl[LR_RANK];
#pragma unroll
    for (int l = 0; l < N; ++l) {
        const double2 v = row ? Ab[l * N + lane] : make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < LR_RANK; ++i) {
            rl[i] = wsum2(make_double2(q[i].x * v.x + q[i].y * v.y, q[i].x * v.y - q[i].y * v.x));
            if (lane == 0) R[i * N + l] = rl[i];
        }
        double2 e = v;
#pragma unroll
        for (int i = 0; i < LR_RANK; ++i) {
            e.x -= q[i].x * rl[i].x - q[i].y * rl[i].y;
            e.y -= q[i].x * rl[i].y + q[i].y * rl[i].x;
        }
        err2 += e.x * e.x + e.y * e.y;
    }
    err2 = wsum(err2);
    if (lane == 0 && anorm2 > 0.0) {
        const double rel = sqrt(err2 / anorm2);
        atomicMax(maxerr, (unsigned long long)__double_as_longlong(rel));  // non-negative doubles order as integers
    }
}

// y = A x (or sigma3^ A sigma3^ x, or b - A x) with the factored hop blocks;
// one thread per dof row k of a site, LR_SPB sites per block.  Threads k < 16
// of a site form t = R x_nbr for direction 1 + k / 4, rank index k % 4.
template <typename T>
__global__ void __launch_bounds__(LR_SPB* N) k_stencil_lr(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                         const C2<T>* __restrict__ F, const C2<T>* __restrict__ b,
                                                         int Nx, int Nt, int dagger, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> xs[LR_SPB][5][N];
    __shared__ C2<T> ts[LR_SPB][4][LR_RANK];
    const int ls = threadIdx.x / N, k = threadIdx.x - ls * N;
    const long s = (long)blockIdx.x * LR_SPB + ls;
    const long nsite = (long)Nx * Nt;
    const bool valid = s < nsite;
    const bool flip = dagger && (k >= N / 2);
    if (valid) {
        const int xx = (int)(s % Nx), t = (int)(s / Nx);
        const long nb[5] = {s, (xx + 1 == Nx) ? s - xx : s + 1, (xx == 0) ? s + Nx - 1 : s - 1,
                            (t + 1 == Nt) ? (long)xx : s + Nx, (t == 0) ? s + (long)Nx * (Nt - 1) : s - Nx};
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const C2<T> v = x[nb[d] * N + k];
            xs[ls][d][k] = flip ? cneg(v) : v;
        }
    }
    __syncthreads();
    const C2<T>* Fs = F + (valid ? s : 0) * (long)LR_SITE;
    if (valid && k < 4 * LR_RANK) {
        const int d = k / LR_RANK, i = k - d * LR_RANK;
        const C2<T>* Rr = Fs + N * N + d * LR_BLOCK + LR_RANK * N + i * N;
        C2<T> tv = mk<T>(0, 0);
#pragma unroll 8
        for (int l = 0; l < N; ++l) tv = cfma(Rr[l], xs[ls][d + 1][l], tv);
        ts[ls][d][i] = tv;
    }
    C2<T> acc = mk<T>(0, 0);
    if (valid) {
#pragma unroll 12
        for (int l = 0; l < N; ++l) acc = cfma(Fs[l * N + k], xs[ls][0][l], acc);
    }
    __syncthreads();
    if (!valid) return;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const C2<T>* Qd = Fs + N * N + d * LR_BLOCK;
#pragma unroll
        for (int i = 0; i < LR_RANK; ++i) acc = cfma(Qd[i * N + k], ts[ls][d][i], acc);
    }
    if (flip) acc = cneg(acc);
    if (b) acc = csub(b[s * N + k], acc);
    y[s * N + k] = acc;
}


// FP32 (bound by HBM): one thread per PAIR of dof rows (12 per site), so every
// operator load is a 16-byte vector of two rows (Q, the self block) or two
// columns (R); sites spread evenly over one block per SM and wave, as in the
// dense FP32 stencil.  The 16 inner products t = R x_nbr of a site are formed
// from per-thread partial sums (two entries each) added in shared memory in a
// fixed order.
constexpr int LRF_TPS = 12;
constexpr int LRF_MAX_SPB = 16;  // sites per block (the partial sums need 24.6 KB of shared memory)

__global__ void __launch_bounds__(LRF_MAX_SPB* LRF_TPS) k_stencil_lr_f32(float2* __restrict__ y,
                                                                         const float2* __restrict__ x,
                                                                         const float2* __restrict__ F,
                                                                         const float2* __restrict__ b, int Nx,
                                                                         int Nt, int spb, int dagger, Gate g) {
    if (!gate_open(g)) return;
    __shared__ float4 xs[LRF_MAX_SPB][5][N / 2];
    __shared__ float2 part[LRF_MAX_SPB][4 * LR_RANK][LRF_TPS];
    __shared__ float2 ts[LRF_MAX_SPB][4 * LR_RANK];
    const int ls = threadIdx.x / LRF_TPS, kt = threadIdx.x - ls * LRF_TPS;
    const long s = (long)blockIdx.x * spb + ls;
    const long nsite = (long)Nx * Nt;
    const bool valid = ls < spb && s < nsite;
    const bool flip = dagger && (2 * kt >= N / 2);
    const float4* F4 = reinterpret_cast<const float4*>(F + (valid ? s : 0) * (long)LR_SITE);
    float4 a[N];
    if (valid) {
#pragma unroll
        for (int l = 0; l < N; ++l) a[l] = __ldg(F4 + l * (N / 2) + kt);  // self block, rows 2 kt, 2 kt + 1
        const int xx = (int)(s % Nx), t = (int)(s / Nx);
        const long nb[5] = {s, (xx + 1 == Nx) ? s - xx : s + 1, (xx == 0) ? s + Nx - 1 : s - 1,
                            (t + 1 == Nt) ? (long)xx : s + Nx, (t == 0) ? s + (long)Nx * (Nt - 1) : s - Nx};
        const float4* x4 = reinterpret_cast<const float4*>(x);
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            float4 v = __ldg(x4 + nb[d] * (N / 2) + kt);
            if (flip) v = make_float4(-v.x, -v.y, -v.z, -v.w);
            xs[ls][d][kt] = v;
        }
    }
    __syncthreads();
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    if (valid) {
        // partial sums of t_{d,i} over columns 2 kt, 2 kt + 1
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const float4 xv = xs[ls][d + 1][kt];
            const float4* R4 = F4 + (N * N + d * LR_BLOCK + LR_RANK * N) / 2;
#pragma unroll
            for (int i = 0; i < LR_RANK; ++i) {
                const float4 r = __ldg(R4 + i * (N / 2) + kt);
                float2 p = cfma(make_float2(r.x, r.y), make_float2(xv.x, xv.y), make_float2(0.f, 0.f));
                p = cfma(make_float2(r.z, r.w), make_float2(xv.z, xv.w), p);
                part[ls][d * LR_RANK + i][kt] = p;
            }
        }
        const float2* xsl = reinterpret_cast<const float2*>(&xs[ls][0][0]);
#pragma unroll
        for (int l = 0; l < N; ++l) {
            const float2 xv = xsl[l];
            acc0 = cfma(make_float2(a[l].x, a[l].y), xv, acc0);
            acc1 = cfma(make_float2(a[l].z, a[l].w), xv, acc1);
        }
    }
    __syncthreads();
    if (valid) {
        for (int q = kt; q < 4 * LR_RANK; q += LRF_TPS) {
            float2 tv = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < LRF_TPS; ++j) {
                tv.x += part[ls][q][j].x;
                tv.y += part[ls][q][j].y;
            }
            ts[ls][q] = tv;
        }
    }
    __syncthreads();
    if (!valid) return;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const float4* Q4 = F4 + (N * N + d * LR_BLOCK) / 2;
#pragma unroll
        for (int i = 0; i < LR_RANK; ++i) {
            const float4 q = __ldg(Q4 + i * (N / 2) + kt);
            const float2 tv = ts[ls][d * LR_RANK + i];
            acc0 = cfma(make_float2(q.x, q.y), tv, acc0);
            acc1 = cfma(make_float2(q.z, q.w), tv, acc1);
        }
    }
    if (flip) {
        acc0 = cneg(acc0);
        acc1 = cneg(acc1);
    }
    if (b) {
        const float4 bv = __ldg(reinterpret_cast<const float4*>(b) + s * (N / 2) + kt);
        acc0 = make_float2(bv.x - acc0.x, bv.y - acc0.y);
        acc1 = make_float2(bv.z - acc1.x, bv.w - acc1.y);
    }
    reinterpret_cast<float4*>(y)[s * (N / 2) + kt] = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
}

}  // namespace

template <typename T>
void launch_stencil_lr(C2<T>* y, const C2<T>* x, const C2<T>* F, const C2<T>* b, int Nx, int Nt, bool dagger,
                       Gate g, cudaStream_t s, int shape) {
    const long nsite = (long)Nx * Nt;
    if constexpr (std::is_same<T, float>::value) {
        // built-in shape: whole waves of one block per SM, sites spread evenly
        // over the blocks; or `shape` sites per block
        const long sms = sm_count();
        const long waves = (nsite + sms * LRF_MAX_SPB - 1) / (sms * LRF_MAX_SPB);
        const long blocks = std::min(sms * waves, nsite);
        const int spb = (shape >= 1 && shape <= LRF_MAX_SPB) ? shape : (int)((nsite + blocks - 1) / blocks);
        const unsigned grid = (unsigned)((nsite + spb - 1) / spb);
        k_stencil_lr_f32<<<grid, spb * LRF_TPS, 0, s>>>(y, x, F, b, Nx, Nt, spb, dagger ? 1 : 0, g);
    } else {
        const unsigned grid = (unsigned)((nsite + LR_SPB - 1) / LR_SPB);
        k_stencil_lr<T><<<grid, LR_SPB * N, 0, s>>>(y, x, F, b, Nx, Nt, dagger ? 1 : 0, g);
    }
    count_launch();
}

void launch_factor_hops(double2* F, const double2* A, long nsite, double* maxerr, cudaStream_t s) {
    cudaMemsetAsync(maxerr, 0, sizeof(double), s);
    const long warps = nsite * 5;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    k_factor_hops<<<grid, 256, 0, s>>>(F, A, nsite, reinterpret_cast<unsigned long long*>(maxerr));
    count_launch();
}

template void launch_stencil_lr<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, int,
                                        int, bool, Gate, cudaStream_t, int);
template void launch_stencil_lr<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, int, int,
                                       bool, Gate, cudaStream_t, int);

}  // namespace mg
