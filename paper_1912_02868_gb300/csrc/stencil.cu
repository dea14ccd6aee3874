// Coarse-grid operators D^ = P^+ D P (Section 2) as 5-point block stencils:
//
//   y(s) = sum_{d in {self, +x, -x, +t, -t}} A[s, d] x(nbr(s, d)),
//
// with dof x dof complex blocks (dof = 24) stored column-major per block,
// A[s][d][l][k] = entry (k, l), so that the dof threads k of one site read one
// contiguous column per step: every block is streamed once per apply, fully
// coalesced.  The five neighbour vectors of a site are staged in shared memory
// and broadcast to its dof threads.  dagger applies sigma3^ A sigma3^ with
// sigma3^ = diag(+1 x dof/2, -1 x dof/2), the adjoint of a Galerkin operator.
//
// FP64 (bound by the FP64 pipe on this GPU): one thread per dof row, 8 sites
// per block.  FP32 (bound by HBM at the intermediate grid): one thread per
// PAIR of dof rows, so every operator load is a 16-byte vector load of two
// rows of one column (a warp reads 512 contiguous bytes), and the sites are
// split evenly over the SMs (one block of up to 32 sites per SM and wave), so
// no SM is left with an extra block at the tail.  The first direction's
// operator loads are issued before the neighbour staging barrier.
#include <algorithm>
#include <type_traits>

#include "ops.cuh"

namespace mg {

namespace {

constexpr int SPB = 8;  // sites per block

template <typename T, int N>
__global__ void __launch_bounds__(SPB* N) k_stencil(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                    const C2<T>* __restrict__ A, const C2<T>* __restrict__ b,
                                                    int Nx, int Nt, int dagger, Gate g) {
    if (!gate_open(g)) return;
    __shared__ C2<T> xs[SPB][5][N];
    const int ls = threadIdx.x / N, k = threadIdx.x - ls * N;
    const long s = (long)blockIdx.x * SPB + ls;
    const long nsite = (long)Nx * Nt;
    const bool valid = s < nsite;
    const bool flip = dagger && (k >= N / 2);
    if (valid) {
        const int xx = (int)(s % Nx), t = (int)(s / Nx);
        const long nb[5] = {s, (xx + 1 == Nx) ? s - xx : s + 1, (xx == 0) ? s + Nx - 1 : s - 1,
                            (t + 1 == Nt) ? (long)xx : s + Nx, (t == 0) ? s + (long)Nx * (Nt - 1) : s - Nx};
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            C2<T> v = x[nb[d] * N + k];
            xs[ls][d][k] = flip ? cneg(v) : v;
        }
    }
    __syncthreads();
    if (!valid) return;
    const C2<T>* Ab = A + s * (5L * N * N) + k;
    C2<T> acc = mk<T>(0, 0);
#pragma unroll
    for (int d = 0; d < 5; ++d) {
#pragma unroll 12
        for (int l = 0; l < N; ++l) acc = cfma(Ab[(d * N + l) * N], xs[ls][d][l], acc);
    }
    if (flip) acc = cneg(acc);
    if (b) acc = csub(b[s * N + k], acc);
    y[s * N + k] = acc;
}

constexpr int F32_TPS = 12;      // threads per site: two dof rows each
constexpr int F32_MAX_SPB = 32;  // sites per block (384 threads)

__global__ void __launch_bounds__(F32_MAX_SPB* F32_TPS) k_stencil_f32(float2* __restrict__ y,
                                                                       const float2* __restrict__ x,
                                                                       const float2* __restrict__ A,
                                                                       const float2* __restrict__ b, int Nx, int Nt,
                                                                       int spb, int dagger, Gate g) {
    constexpr int N = 24;
    if (!gate_open(g)) return;
    __shared__ float4 xs[F32_MAX_SPB][5][N / 2];  // neighbour values, two dofs per entry
    const int ls = threadIdx.x / F32_TPS, kt = threadIdx.x - ls * F32_TPS;
    const long s = (long)blockIdx.x * spb + ls;
    const long nsite = (long)Nx * Nt;
    const bool valid = ls < spb && s < nsite;
    const bool flip = dagger && (2 * kt >= N / 2);
    // rows 2 kt, 2 kt + 1 of column l of block d: A4[(d * N + l) * (N / 2) + kt]
    const float4* A4 = reinterpret_cast<const float4*>(A + (valid ? s : 0) * (5L * N * N)) + kt;
    float4 a[N];
    if (valid) {
#pragma unroll
        for (int l = 0; l < N; ++l) a[l] = __ldg(A4 + l * (N / 2));
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
    if (!valid) return;
    const float2* xsl = reinterpret_cast<const float2*>(&xs[ls][0][0]);
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        if (d > 0) {
#pragma unroll
            for (int l = 0; l < N; ++l) a[l] = __ldg(A4 + (d * N + l) * (N / 2));
        }
#pragma unroll
        for (int l = 0; l < N; ++l) {
            const float2 xv = xsl[d * N + l];
            acc0 = cfma(make_float2(a[l].x, a[l].y), xv, acc0);
            acc1 = cfma(make_float2(a[l].z, a[l].w), xv, acc1);
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
void launch_stencil(C2<T>* y, const C2<T>* x, const C2<T>* A, const C2<T>* b, int Nx, int Nt, int dof,
                    bool dagger, Gate g, cudaStream_t s, int shape) {
    const long nsite = (long)Nx * Nt;
    // only dof = 24 is built (12 near-null vectors, chirally doubled)
    if constexpr (std::is_same<T, float>::value) {
        // built-in shape: whole waves of one block per SM, sites spread evenly
        // over the blocks; or `shape` sites per block
        const long sms = sm_count();
        const long waves = (nsite + sms * F32_MAX_SPB - 1) / (sms * F32_MAX_SPB);
        const long blocks = std::min(sms * waves, nsite);
        const int spb = (shape >= 1 && shape <= F32_MAX_SPB) ? shape : (int)((nsite + blocks - 1) / blocks);
        const unsigned grid = (unsigned)((nsite + spb - 1) / spb);
        k_stencil_f32<<<grid, spb * F32_TPS, 0, s>>>(y, x, A, b, Nx, Nt, spb, dagger ? 1 : 0, g);
    } else {
        const unsigned grid = (unsigned)((nsite + SPB - 1) / SPB);
        k_stencil<T, 24><<<grid, SPB * 24, 0, s>>>(y, x, A, b, Nx, Nt, dagger ? 1 : 0, g);
    }
    count_launch();
}

template void launch_stencil<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, int, int,
                                     int, bool, Gate, cudaStream_t, int);
template void launch_stencil<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, int, int, int,
                                    bool, Gate, cudaStream_t, int);

}  // namespace mg
