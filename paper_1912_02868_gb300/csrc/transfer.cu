// Restriction P^+ and prolongation P between grids (Section 2: the columns of
// P are the chirally doubled near-null vectors, blocked on 4^2 sites and
// orthonormalised per block and chirality).
//
// Q[B][c][j][l][a]: coarse site B, chirality c, vector j < 12, finer site
// l = lx + 4 lt of the 4x4 block, dof a < h of chirality c at that site
// (h = 1 on the fine grid, 12 on the intermediate grid).  Coarse dof k = 12c + j.
//   restrict:  v^[B][k]           = sum_{l,a} conj(Q[B][c][j][l][a]) v[s(B,l)][c h + a]
//   prolong:   v[s(B,l)][c h + a] = sum_j Q[B][c][j][l][a] v^[B][12 c + j]
#include "batch.cuh"

namespace mg {

namespace {

constexpr int NV = 12;      // near-null vectors per chirality
constexpr int BL = 4;       // block extent
constexpr int BS = BL * BL; // sites per block

// one CTA per coarse site, one warp per coarse dof (strided), lanes over the
// 16 h entries of that column of P.
// blockIdx.y = right-hand side r of a batch (vectors at r * cr and r * fr, gate r)
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(C2<T>* __restrict__ vc, const C2<T>* __restrict__ v,
                                                  const C2<T>* __restrict__ Q, int NxF, int h, long cr, long fr,
                                                  Gate g) {
    const int rb = blockIdx.y;
    if (!gate_open(g, rb)) return;
    vc += rb * cr;
    v += rb * fr;
    const int B = blockIdx.x;
    const int NxC = NxF / BL;
    const int bx = B % NxC, bt = B / NxC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int len = BS * h;
    for (int k = warp; k < 2 * NV; k += nw) {
        const int c = k / NV;
        const C2<T>* q = Q + ((long)B * 2 * NV + k) * len;
        C2<T> acc = mk<T>(0, 0);
        for (int e = lane; e < len; e += 32) {
            const int l = e / h, a = e - l * h;
            const long fs = (long)(bt * BL + l / BL) * NxF + bx * BL + (l % BL);
            acc = cfmac(q[e], v[fs * 2 * h + c * h + a], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) vc[(long)B * 2 * NV + k] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong(C2<T>* __restrict__ v, const C2<T>* __restrict__ vc,
                                                 const C2<T>* __restrict__ Q, int NxF, int NtF, int h, int accumulate,
                                                 long fr, long cr, Gate g) {
    const int rb = blockIdx.y;
    if (!gate_open(g, rb)) return;
    v += rb * fr;
    vc += rb * cr;
    const long nf = (long)NxF * NtF * 2 * h;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nf) return;
    const long fs = e / (2 * h);
    const int r = (int)(e - fs * 2 * h);
    const int c = r / h, a = r - c * h;
    const int xf = (int)(fs % NxF), tf = (int)(fs / NxF);
    const int B = (tf / BL) * (NxF / BL) + xf / BL;
    const int l = (xf % BL) + BL * (tf % BL);
    const C2<T>* q = Q + (((long)B * 2 * NV + c * NV) * BS + l) * h + a;
    const C2<T>* w = vc + (long)B * 2 * NV + c * NV;
    C2<T> acc = accumulate ? v[e] : mk<T>(0, 0);
#pragma unroll
    for (int j = 0; j < NV; ++j) acc = cfma(q[(long)j * BS * h], w[j], acc);
    v[e] = acc;
}

}  // namespace

template <typename T>
void launch_brestrict(C2<T>* coarse, long cr, const C2<T>* fine, long fr, const C2<T>* Q, int NxF, int NtF, int h,
                      int nb, Gate g, cudaStream_t s) {
    const int nc = (NxF / BL) * (NtF / BL);
    k_restrict<T><<<dim3(nc, nb), 256, 0, s>>>(coarse, fine, Q, NxF, h, cr, fr, g);
    count_launch();
}

template <typename T>
void launch_bprolong(C2<T>* fine, long fr, const C2<T>* coarse, long cr, const C2<T>* Q, int NxF, int NtF, int h,
                     bool accumulate, int nb, Gate g, cudaStream_t s) {
    const long nf = (long)NxF * NtF * 2 * h;
    k_prolong<T><<<dim3(nblocks(nf, 256), nb), 256, 0, s>>>(fine, coarse, Q, NxF, NtF, h, accumulate ? 1 : 0, fr, cr,
                                                              g);
    count_launch();
}

template <typename T>
void launch_restrict(C2<T>* coarse, const C2<T>* fine, const C2<T>* Q, int NxF, int NtF, int h, Gate g,
                     cudaStream_t s) {
    launch_brestrict<T>(coarse, 0, fine, 0, Q, NxF, NtF, h, 1, g, s);
}

template <typename T>
void launch_prolong(C2<T>* fine, const C2<T>* coarse, const C2<T>* Q, int NxF, int NtF, int h, bool accumulate,
                    Gate g, cudaStream_t s) {
    launch_bprolong<T>(fine, 0, coarse, 0, Q, NxF, NtF, h, accumulate, 1, g, s);
}

template void launch_restrict<double>(C2<double>*, const C2<double>*, const C2<double>*, int, int, int, Gate,
                                      cudaStream_t);
template void launch_restrict<float>(C2<float>*, const C2<float>*, const C2<float>*, int, int, int, Gate,
                                     cudaStream_t);
template void launch_prolong<double>(C2<double>*, const C2<double>*, const C2<double>*, int, int, int, bool, Gate,
                                     cudaStream_t);
template void launch_prolong<float>(C2<float>*, const C2<float>*, const C2<float>*, int, int, int, bool, Gate,
                                    cudaStream_t);
template void launch_brestrict<double>(C2<double>*, long, const C2<double>*, long, const C2<double>*, int, int, int,
                                       int, Gate, cudaStream_t);
template void launch_brestrict<float>(C2<float>*, long, const C2<float>*, long, const C2<float>*, int, int, int, int,
                                      Gate, cudaStream_t);
template void launch_bprolong<double>(C2<double>*, long, const C2<double>*, long, const C2<double>*, int, int, int,
                                      bool, int, Gate, cudaStream_t);
template void launch_bprolong<float>(C2<float>*, long, const C2<float>*, long, const C2<float>*, int, int, int, bool,
                                     int, Gate, cudaStream_t);

}  // namespace mg
