// Fine-grid Wilson-Dirac operator of the 2D Schwinger model (Section 2):
//
//   (D psi)(s) = (m0 + 2) psi(s)
//              - 1/2 sum_mu [ (1 - sigma_mu) U_mu(s) psi(s + mu)
//                           + (1 + sigma_mu) U_mu(s - mu)^* psi(s - mu) ]
//
// sigma_1 on x, sigma_2 on t, periodic in x, antiperiodic in t (a hop across
// t = L_t - 1 <-> 0 carries -1).  D^+ = sigma_3 D sigma_3.
//
// Each (1 -/+ sigma_mu) has rank one, so a hop moves one complex number h:
//   +x: h = U_x(s)   (p0 - p1),        contributes (-h/2, +h/2)
//   -x: h = U_x^*(s-x)(p0 + p1),       contributes (-h/2, -h/2)
//   +t: h = U_t(s)   (p0 + i p1),      contributes (-h/2, +i h/2)
//   -t: h = U_t^*(s-t)(p0 - i p1),     contributes (-h/2, -i h/2)
// One thread per site; the site's two spin components and its two links are
// one 32-byte (FP64) or 16-byte (FP32) vector load each.  Neighbour spinors are
// re-read by four threads and come from L1/L2; at 1024^2 the working set
// (2 spinor fields + gauge) stays resident in the 129 MB L2 between applies.
#include "batch.cuh"

namespace mg {

namespace {

template <typename T> struct alignas(2 * sizeof(C2<T>)) Pair {
    C2<T> a, b;
};

template <typename T, bool DAG>
__device__ __forceinline__ void load_site(const C2<T>* __restrict__ x, int s, C2<T>& p0, C2<T>& p1) {
    const Pair<T> v = reinterpret_cast<const Pair<T>*>(x)[s];
    p0 = v.a;
    p1 = DAG ? cneg(v.b) : v.b;
}

// blockIdx.y = right-hand side r of a batch: vectors at offset r * vr, gate r
template <typename T, bool DAG, bool RES>
__global__ void __launch_bounds__(256) k_wilson(C2<T>* __restrict__ y, const C2<T>* __restrict__ x,
                                                const C2<T>* __restrict__ U, const C2<T>* __restrict__ b,
                                                T diag, int Lx, int Lt, long vr, Gate g) {
    const int rb = blockIdx.y;
    if (!gate_open(g, rb)) return;
    y += rb * vr;
    x += rb * vr;
    if (RES) b += rb * vr;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Lx * Lt) return;
    const int xx = s % Lx, t = s / Lx;
    const int sxp = (xx + 1 == Lx) ? s - xx : s + 1;
    const int sxm = (xx == 0) ? s + Lx - 1 : s - 1;
    const int stp = (t + 1 == Lt) ? xx : s + Lx;
    const int stm = (t == 0) ? s + Lx * (Lt - 1) : s - Lx;
    const T sf = (t + 1 == Lt) ? T(-1) : T(1);
    const T sb = (t == 0) ? T(-1) : T(1);

    const Pair<T>* U2 = reinterpret_cast<const Pair<T>*>(U);
    const Pair<T> us = U2[s];
    const C2<T> uxm = U2[sxm].a;
    const C2<T> utm = U2[stm].b;

    C2<T> p0, p1, q0, q1;
    load_site<T, DAG>(x, s, p0, p1);
    // sum of the hops before the factor -1/2: spin 0 and spin 1 parts
    C2<T> a0, a1, h;
    // +x
    load_site<T, DAG>(x, sxp, q0, q1);
    h = cmul(us.a, csub(q0, q1));
    a0 = h;
    a1 = cneg(h);
    // -x
    load_site<T, DAG>(x, sxm, q0, q1);
    h = cmulc(uxm, cadd(q0, q1));
    a0 = cadd(a0, h);
    a1 = cadd(a1, h);
    // +t
    load_site<T, DAG>(x, stp, q0, q1);
    h = cscale(cmul(us.b, cadd(q0, cmuli(q1))), sf);
    a0 = cadd(a0, h);
    a1 = csub(a1, cmuli(h));
    // -t
    load_site<T, DAG>(x, stm, q0, q1);
    h = cscale(cmulc(utm, csub(q0, cmuli(q1))), sb);
    a0 = cadd(a0, h);
    a1 = cadd(a1, cmuli(h));

    C2<T> o0, o1;
    o0.x = diag * p0.x - T(0.5) * a0.x;
    o0.y = diag * p0.y - T(0.5) * a0.y;
    o1.x = diag * p1.x - T(0.5) * a1.x;
    o1.y = diag * p1.y - T(0.5) * a1.y;
    if (DAG) o1 = cneg(o1);
    if (RES) {
        const Pair<T> bb = reinterpret_cast<const Pair<T>*>(b)[s];
        o0 = csub(bb.a, o0);
        o1 = csub(bb.b, o1);
    }
    Pair<T> out;
    out.a = o0;
    out.b = o1;
    reinterpret_cast<Pair<T>*>(y)[s] = out;
}

}  // namespace

// threads: threads per block, one thread per site (a multiple of 32, at most 256)
template <typename T>
void wilson_grid(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt, bool dagger,
                 long vr, int nb, Gate g, cudaStream_t s, int threads = 256) {
    const int n = Lx * Lt;
    const dim3 grid(nblocks(n, threads), nb);
    const T diag = (T)(m0 + 2.0);
    if (dagger) {
        if (b) k_wilson<T, true, true><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson<T, true, false><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    } else {
        if (b) k_wilson<T, false, true><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
        else k_wilson<T, false, false><<<grid, threads, 0, s>>>(y, x, U, b, diag, Lx, Lt, vr, g);
    }
    count_launch();
}

template <typename T>
void launch_wilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt,
                   bool dagger, Gate g, cudaStream_t s, int shape) {
    const int threads = (shape >= 32 && shape <= 256 && shape % 32 == 0) ? shape : 256;
    wilson_grid<T>(y, x, U, b, m0, Lx, Lt, dagger, 0, 1, g, s, threads);
}

template <typename T>
void launch_bwilson(C2<T>* y, const C2<T>* x, const C2<T>* U, const C2<T>* b, double m0, int Lx, int Lt, long vr,
                    int nb, Gate g, cudaStream_t s) {
    wilson_grid<T>(y, x, U, b, m0, Lx, Lt, false, vr, nb, g, s);
}

template void launch_wilson<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, double,
                                    int, int, bool, Gate, cudaStream_t, int);
template void launch_wilson<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, double, int,
                                   int, bool, Gate, cudaStream_t, int);
template void launch_bwilson<double>(C2<double>*, const C2<double>*, const C2<double>*, const C2<double>*, double,
                                     int, int, long, int, Gate, cudaStream_t);
template void launch_bwilson<float>(C2<float>*, const C2<float>*, const C2<float>*, const C2<float>*, double, int,
                                    int, long, int, Gate, cudaStream_t);

}  // namespace mg
