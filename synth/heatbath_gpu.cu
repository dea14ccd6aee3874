/*
 * The seeded U(1) heatbath of heatbath.c on the GPU, bit-identical to it.
 *
 * Input generator only: no solver arithmetic.  Same action, sweep order
 * (checkerboard, direction x first, then t, cold start), counter-based random
 * numbers keyed by (seed, sweep, direction, link, attempt), and the same
 * floating-point operations in the same order: +, -, *, /, sqrt and ldexp,
 * each correctly rounded in FP64, and no contraction into FMA (the file is
 * compiled with -fmad=false).  A sub-sweep (one direction, one parity) updates
 * links that share no staple, one thread per link, so the order of the updates
 * inside it does not matter and the result equals the host generator's.
 *
 * The rejection loop of the von Mises draw is bounded: after HB_MAX_ATTEMPTS
 * rejections of one draw (acceptance is above one half per attempt, so this
 * does not happen) the link is left unchanged and an error counter is raised,
 * which the host turns into a failed call.
 *
 * Layout: double[L_t][L_x][2 (mu)][2 (re, im)] in device memory.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#define HB_MAX_ATTEMPTS 65536

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t key, uint64_t ctr) {
    const uint64_t z = mix64(key ^ mix64(ctr));
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// the host generator's arithmetic-only exponential (Cody-Waite reduction,
// Taylor series to r^17), operation for operation
__device__ double det_exp(double x) {
    if (x < -745.0) return 0.0;
    if (x > 709.0) return __longlong_as_double(0x7FF0000000000000LL);
    const double ln2_hi = 6.93147180369123816490e-01;
    const double ln2_lo = 1.90821492927058770002e-10;
    const double inv_ln2 = 1.44269504088896338700e+00;
    const double t = x * inv_ln2;
    const double n = (t >= 0.0) ? (double)(long long)(t + 0.5) : -(double)(long long)(0.5 - t);
    const double r = (x - n * ln2_hi) - n * ln2_lo;
    double p = 1.0;
    for (int k = 17; k >= 1; --k) p = 1.0 + p * r / (double)k;
    return ldexp(p, (int)n);
}

// Best-Fisher von Mises draw around angle 0 as (cos, sin); false if the
// attempt bound ran out
__device__ bool vonmises(double kappa, uint64_t key, uint64_t ctr0, double* c_out, double* s_out) {
    if (kappa < 1e-8) {
        for (uint64_t att = 0; att < HB_MAX_ATTEMPTS; ++att) {
            const double a = 2.0 * uniform01(key, ctr0 + 8 * att) - 1.0;
            const double b = 2.0 * uniform01(key, ctr0 + 8 * att + 1) - 1.0;
            const double q = a * a + b * b;
            if (q > 0.0 && q <= 1.0) {
                *c_out = (a * a - b * b) / q;
                *s_out = 2.0 * a * b / q;
                return true;
            }
        }
        return false;
    }
    const double tau = 1.0 + sqrt(1.0 + 4.0 * kappa * kappa);
    const double rho = (tau - sqrt(2.0 * tau)) / (2.0 * kappa);
    const double r = (1.0 + rho * rho) / (2.0 * rho);
    for (uint64_t att = 0; att < HB_MAX_ATTEMPTS; ++att) {
        const uint64_t c = ctr0 + 8 * att;
        const double a = 2.0 * uniform01(key, c) - 1.0;
        const double b = 2.0 * uniform01(key, c + 1) - 1.0;
        const double q = a * a + b * b;
        if (!(q > 0.0 && q <= 1.0)) continue;
        const double z = (a * a - b * b) / q;
        const double f = (1.0 + r * z) / (r + z);
        const double cc = kappa * (r - f);
        const double u2 = uniform01(key, c + 2);
        bool accept = (cc * (2.0 - cc) - u2 > 0.0);
        if (!accept) accept = (cc >= u2 * det_exp(cc - 1.0));
        if (!accept) continue;
        const double u3 = uniform01(key, c + 3);
        double s = 1.0 - f * f;
        s = (s > 0.0) ? sqrt(s) : 0.0;
        *c_out = f;
        *s_out = (u3 < 0.5) ? -s : s;
        return true;
    }
    return false;
}

__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double* cr, double* ci) {
    const double pr = ar * br;
    const double qr = ai * bi;
    const double pi = ar * bi;
    const double qi = ai * br;
    *cr = pr - qr;
    *ci = pi + qi;
}

__global__ void k_cold(double* U, long nlinks) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nlinks) {
        U[2 * i] = 1.0;
        U[2 * i + 1] = 0.0;
    }
}

// one sub-sweep: the links of direction mu on sites of parity par
__global__ void k_subsweep(double* U, int Lx, int Lt, double beta, int sw, int mu, int par, uint64_t key,
                           unsigned* err) {
    const long half = (long)Lx * Lt / 2;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const int hx = Lx / 2;
    const int t = (int)(i / hx);
    const int x = 2 * (int)(i % hx) + ((par + t) & 1);
    const long s = (long)t * Lx + x;
    const int xp = (x + 1) % Lx, xm = (x + Lx - 1) % Lx;
    const int tp = (t + 1) % Lt, tm = (t + Lt - 1) % Lt;
#define LNK(xx, tt, m, ri) U[(((long)(tt) * Lx + (xx)) * 2 + (m)) * 2 + (ri)]
    double ar, ai, pr, pi_, qr, qi;
    if (mu == 0) {
        cmul(LNK(xp, t, 1, 0), LNK(xp, t, 1, 1), LNK(x, tp, 0, 0), -LNK(x, tp, 0, 1), &pr, &pi_);
        cmul(pr, pi_, LNK(x, t, 1, 0), -LNK(x, t, 1, 1), &ar, &ai);
        cmul(LNK(x, tm, 0, 0), -LNK(x, tm, 0, 1), LNK(xp, tm, 1, 0), -LNK(xp, tm, 1, 1), &pr, &pi_);
        cmul(pr, pi_, LNK(x, tm, 1, 0), LNK(x, tm, 1, 1), &qr, &qi);
    } else {
        cmul(LNK(x, tp, 0, 0), LNK(x, tp, 0, 1), LNK(xp, t, 1, 0), -LNK(xp, t, 1, 1), &pr, &pi_);
        cmul(pr, pi_, LNK(x, t, 0, 0), -LNK(x, t, 0, 1), &ar, &ai);
        cmul(LNK(xm, tp, 0, 0), -LNK(xm, tp, 0, 1), LNK(xm, t, 1, 0), -LNK(xm, t, 1, 1), &pr, &pi_);
        cmul(pr, pi_, LNK(xm, t, 0, 0), LNK(xm, t, 0, 1), &qr, &qi);
    }
    ar = ar + qr;
    ai = ai + qi;
    const double n2 = ar * ar + ai * ai;
    const double nrm = sqrt(n2);
    double c, sn;
    const uint64_t ctr = ((((uint64_t)sw * 2u + (uint64_t)mu) << 24) | (uint64_t)s) << 24;
    if (!vonmises(beta * nrm, key, ctr, &c, &sn)) {
        atomicAdd(err, 1u);
        return;
    }
    double ur, ui;
    if (nrm > 0.0) {
        cmul(c, sn, ar / nrm, -ai / nrm, &ur, &ui);
    } else {
        ur = c;
        ui = sn;
    }
    LNK(x, t, mu, 0) = ur;
    LNK(x, t, mu, 1) = ui;
#undef LNK
}

uint64_t host_mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

/* Fill the device array U with the field synth_heatbath would produce for the
 * same arguments, on `stream` (synchronised before returning).  Returns 0 on
 * success, -1 on invalid arguments, -2 on a CUDA error, -3 if a von Mises draw
 * ran out of attempts. */
extern "C" int synth_heatbath_gpu(double* U, int Lx, int Lt, double beta, int sweeps, uint64_t seed,
                                  void* stream) {
    if (!U || Lx < 2 || Lt < 2 || (Lx & 1) || (Lt & 1) || sweeps < 0 || sweeps >= (1 << 14) || beta < 0.0 ||
        (long)Lx * Lt >= (1L << 24))
        return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long V = (long)Lx * Lt;
    const uint64_t key = host_mix64(seed ^ 0x5CA1AB1E0DDBA11ULL);
    unsigned* err = nullptr;
    if (cudaMallocAsync(&err, sizeof(unsigned), s) != cudaSuccess) return -2;
    cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    const int threads = 256;
    k_cold<<<(unsigned)((2 * V + threads - 1) / threads), threads, 0, s>>>(U, 2 * V);
    const unsigned blocks = (unsigned)((V / 2 + threads - 1) / threads);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int mu = 0; mu < 2; ++mu)
            for (int par = 0; par < 2; ++par) k_subsweep<<<blocks, threads, 0, s>>>(U, Lx, Lt, beta, sw, mu, par, key, err);
    unsigned herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -2;
    return herr ? -3 : 0;
}
