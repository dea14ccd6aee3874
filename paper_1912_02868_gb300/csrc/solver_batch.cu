// Lockstep solve of a block of right-hand sides of one operator (Section 2's
// method for many b with the same D): one FGMRES(8) per right-hand side in
// FP64, advanced one outer step at a time for the whole block, preconditioned
// by one batched V-cycle.  Every kernel of a step runs all right-hand sides of
// the block in one launch; per-right-hand-side gates skip those whose cycle has
// stopped.  On the intermediate and coarsest grids the 24 x 24 block products
// run on tensor cores (BF16 or FP16 operator, FP32 vectors split in two 16-bit
// parts, FP32 accumulation), so one pass over an operator block serves eight
// right-hand sides per MMA tile.  The coarsest solves of a step are one batched
// GMRES-Proj (the deflation space shared by all right-hand sides, Section 2),
// whose cycles are enqueued whole and whose host loop reads one count per
// cycle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "coarse_block.cuh"
#include "handle.cuh"

namespace mg {

namespace {

constexpr int NSC = 8;  // per-right-hand-side scalars: fnb2, r2, level-norm, cnb2, cr2

// scalars of right-hand side 0 (stride NSC)
enum { SC_FNB2 = 0, SC_R2 = 1, SC_LVL = 2, SC_CNB2 = 3, SC_CR2 = 4 };

// gather the step gates of a block's Krylov states for one read by the host
__global__ void k_gather_gates(int* out, const KState* ks, int nb) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nb) out[r] = ks[r].step_gate;
}

__global__ void k_gate_to_flags(int* flags, Gate g, int nb) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nb) flags[r] = gate_open(g, r) ? 1 : 0;
}

// after a coarse GMRES-Proj cycle: iterations, and right-hand side r stays
// active while its cycle did not converge and the cycle limit is not reached;
// *count = right-hand sides still active; *cycles counts the cycles run
__global__ void k_coarse_cycle_end(int* cact, long long* citers, const KState* cks, int nb, int* cycles,
                                   int max_cycles, int* count) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int done = *cycles + 1;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        if (!cact[r]) continue;
        citers[r] += cks[r].j;
        const int on = (!cks[r].conv && done < max_cycles) ? 1 : 0;
        cact[r] = on;
        if (on) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *count = cnt;
        *cycles = done;
    }
}

}  // namespace

struct BatchWS {
    int nbp = 0;
    int fp16 = -1;               // format of Af (-1: not built)
    unsigned* Af[3] = {nullptr, nullptr, nullptr};
    double2 *fV = nullptr, *fZ = nullptr, *fx = nullptr, *fr = nullptr, *fb = nullptr;
    KState* fks = nullptr;
    float2 *v32 = nullptr, *z32 = nullptr;
    struct BL {
        float2 *x = nullptr, *f = nullptr, *r = nullptr, *sV = nullptr;
        KState* ks = nullptr;
    } L[2];
    float2 *f2 = nullptr, *x2 = nullptr;
    float2 *cV = nullptr, *cr = nullptr;
    KState* cks = nullptr;
    double2 *cg = nullptr, *cd = nullptr, *cu = nullptr;
    int* cact = nullptr;
    long long* citers = nullptr;
    int* count = nullptr;
    int* ccycles = nullptr;      // coarse cycles run by the current solve
    int* cgb = nullptr;          // [2][nbp] coarse step gates by step parity
    float2 *cp1 = nullptr, *cp2 = nullptr;  // fused-step partial sums
    float2 *ch1 = nullptr, *ch2 = nullptr;  // fused-step reduced products
    unsigned* ctk = nullptr;                // fused-step tickets
    unsigned* cbar = nullptr;               // tile barriers of the cycle kernel
    bool no_coop = false;                   // the cycle kernel could not be captured: use the step kernels
    int probe = 0;                          // coarse test probe (mg_coarse_solve): a wait that gives up
    long spin = 0;                          // polls of a tile barrier before it gives up (0: default)
    long cp_cap = 0;             // entries of cp1 / cp2
    // the captured coarse cycle: graph, its key, and its kernel count
    cudaGraphExec_t cyc_exec = nullptr;
    int cyc_nb = 0, cyc_k = 0, cyc_fp16 = -1, cyc_coop = -1, cyc_probe = -1;
    long cyc_spin = -1;
    double cyc_tol = 0.0;
    unsigned long long cyc_kernels = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int* oflags = nullptr;       // [nbp] right-hand sides of the block still solving (host-set)
    int* gates = nullptr;        // [nbp] gathered step gates
    double* sc = nullptr;
    BRed red;
    void* pin = nullptr;
};

void destroy_batch(BatchWS* B) {
    if (!B) return;
    if (B->cyc_exec) cudaGraphExecDestroy(B->cyc_exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (cudaEvent_t e : B->ev)
        if (e) cudaEventDestroy(e);
    if (B->pin) cudaFreeHost(B->pin);
    delete B;
}

namespace {

mg_status batch_alloc(Handle& H, int nbp, bool fp16, cudaStream_t s) {
    if (!H.bws) {
        H.bws = new (std::nothrow) BatchWS();
        if (!H.bws) return set_error("out of host memory"), MG_ENOMEM;
    }
    BatchWS& B = *H.bws;
    const mg_params& p = H.p;
    if (B.fp16 != (fp16 ? 1 : 0)) {  // tensor-core operator copies of grids 1 and 2
        for (int l = 1; l < 3; ++l) {
            const long ns = (long)H.L64[l].Nx * H.L64[l].Nt;
            if (!B.Af[l]) MG_TRY(halloc_t(H, &B.Af[l], (size_t)ns * 5 * 576));
            launch_pack_frag(B.Af[l], H.A64[l], ns, fp16, s);
        }
        MG_LAUNCH_CHECK();
        B.fp16 = fp16 ? 1 : 0;
    }
    if (B.nbp >= nbp) return MG_OK;
    // (re)allocate the per-right-hand-side workspaces for nbp right-hand sides; the
    // previous, smaller set stays owned by the handle until it is destroyed
    const long n0 = H.L64[0].n, n1 = H.L64[1].n, n2 = H.L64[2].n;
    const int m = p.fgmres_m, st = p.smooth_steps, ms = MSMAX;
    MG_TRY(halloc_t(H, &B.fV, (size_t)(m + 1) * nbp * n0));
    MG_TRY(halloc_t(H, &B.fZ, (size_t)m * nbp * n0));
    MG_TRY(halloc_t(H, &B.fx, (size_t)nbp * n0));
    MG_TRY(halloc_t(H, &B.fr, (size_t)nbp * n0));
    MG_TRY(halloc_t(H, &B.fb, (size_t)nbp * n0));
    MG_TRY(halloc_t(H, &B.fks, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.v32, (size_t)nbp * n0));
    MG_TRY(halloc_t(H, &B.z32, (size_t)nbp * n0));
    const long nl[2] = {n0, n1};
    for (int l = 0; l < 2; ++l) {
        MG_TRY(halloc_t(H, &B.L[l].x, (size_t)nbp * nl[l]));
        MG_TRY(halloc_t(H, &B.L[l].f, (size_t)nbp * nl[l]));
        MG_TRY(halloc_t(H, &B.L[l].r, (size_t)nbp * nl[l]));
        MG_TRY(halloc_t(H, &B.L[l].sV, (size_t)(st + 1) * nbp * nl[l]));
        MG_TRY(halloc_t(H, &B.L[l].ks, (size_t)nbp));
    }
    MG_TRY(halloc_t(H, &B.f2, (size_t)nbp * n2));
    MG_TRY(halloc_t(H, &B.x2, (size_t)nbp * n2));
    MG_TRY(halloc_t(H, &B.cV, (size_t)(ms + 1) * nbp * n2));
    MG_TRY(halloc_t(H, &B.cr, (size_t)nbp * n2));
    MG_TRY(halloc_t(H, &B.cks, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.cg, (size_t)nbp * KLD));
    MG_TRY(halloc_t(H, &B.cd, (size_t)nbp * KLD));
    MG_TRY(halloc_t(H, &B.cu, (size_t)nbp * KLD));
    MG_TRY(halloc_t(H, &B.cact, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.citers, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.count, 2));  // [0] right-hand sides still active, [1] a tile barrier gave up
    MG_CUDA_TRY(cudaMemsetAsync(B.count, 0, 2 * sizeof(int), s));
    MG_TRY(halloc_t(H, &B.ccycles, 1));
    MG_TRY(halloc_t(H, &B.cgb, (size_t)2 * nbp));
    {
        CBArgs g{};
        cb_geometry(g, (long)H.L64[2].Nx * H.L64[2].Nt, nbp);
        B.cp_cap = (long)nbp * CB_PB * CB_MAXCH;
        MG_TRY(halloc_t(H, &B.cp1, (size_t)B.cp_cap));
        MG_TRY(halloc_t(H, &B.cp2, (size_t)B.cp_cap));
        MG_TRY(halloc_t(H, &B.ch1, (size_t)nbp * CB_PB));
        MG_TRY(halloc_t(H, &B.ch2, (size_t)nbp * CB_PB));
        MG_TRY(halloc_t(H, &B.ctk, (size_t)2 * NB_MAX / NB_TILE));
        MG_CUDA_TRY(cudaMemsetAsync(B.ctk, 0, 2 * NB_MAX / NB_TILE * sizeof(unsigned), s));
        MG_TRY(halloc_t(H, &B.cbar, (size_t)2 * NB_MAX / NB_TILE + 1));
        MG_CUDA_TRY(cudaMemsetAsync(B.cbar, 0, (2 * NB_MAX / NB_TILE + 1) * sizeof(unsigned), s));
    }
    MG_TRY(halloc_t(H, &B.oflags, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.gates, (size_t)nbp));
    MG_TRY(halloc_t(H, &B.sc, (size_t)nbp * NSC));
    B.red.max_chunks = 64;
    MG_TRY(halloc_t(H, &B.red.partial, (size_t)NB_MAX * B.red.max_chunks * RED_MAXD));
    MG_TRY(halloc_t(H, &B.red.ticket, (size_t)NB_MAX));
    MG_CUDA_TRY(cudaMemsetAsync(B.red.ticket, 0, NB_MAX * sizeof(unsigned), s));
    MG_CUDA_TRY(cudaMemsetAsync(B.sc, 0, (size_t)nbp * NSC * sizeof(double), s));
    for (KState* k : {B.fks, B.L[0].ks, B.L[1].ks, B.cks}) MG_CUDA_TRY(cudaMemsetAsync(k, 0, nbp * sizeof(KState), s));
    if (!B.pin && cudaMallocHost(&B.pin, 1 << 16) != cudaSuccess) {
        (void)cudaGetLastError();
        B.pin = nullptr;
        return set_error("cudaMallocHost failed"), MG_ENOMEM;
    }
    B.nbp = nbp;
    return MG_OK;
}

// gates of right-hand side r read from an array of KStates
inline Gate step_gate(KState* ks, int jh) { return Gate{MG_DEVF(ks, int, step_gate), jh, KS_INTS}; }
inline Gate scale_gate(KState* ks, int j) { return Gate{MG_DEVF(ks, int, scale_gate), j, KS_INTS}; }

// One Arnoldi step jh of every right-hand side on the rows V[j][r][n]: w = op(V[jh]),
// CGS2, the least-squares update, and the normalisation (batched arnoldi_step).
template <typename T, typename OpFn>
void barnoldi_step(BatchWS& B, OpFn&& op, C2<T>* V, long n, int nb, KState* ks, int jh, cudaStream_t s) {
    const Gate g = step_gate(ks, jh);
    const long row = (long)nb * n;  // stride of one basis index
    C2<T>* w = V + (long)(jh + 1) * row;
    op(w, V + (long)jh * row, g);
    double2* hA = MG_DEVF(ks, double2, hA);
    double2* hB = MG_DEVF(ks, double2, hB);
    launch_bgram<T>(hA, KS_CPLX, V, row, n, jh + 1, nullptr, 0, w, n, n, nb, B.red, g, s);
    launch_baxpy<T>(w, n, V, row, n, jh + 1, nullptr, 0, hA, KS_CPLX, -1.0, false, n, nb, nullptr, 0, B.red, g, s);
    launch_bgram<T>(hB, KS_CPLX, V, row, n, jh + 1, nullptr, 0, w, n, n, nb, B.red, g, s);
    launch_baxpy<T>(w, n, V, row, n, jh + 1, nullptr, 0, hB, KS_CPLX, -1.0, false, n, nb, MG_DEVF(ks, double, hn2),
                    KS_DBLS, B.red, g, s);
    bks_push(ks, nb, jh, s);
    launch_bscale<T>(w, n, w, n, MG_DEVF(ks, double, scale), KS_DBLS, n, nb, scale_gate(ks, jh + 1), s);
}

// The tensor-core stencil of grid l (1 or 2) for the block: y = A x, or b - A x
void bapply_mma(Handle& H, int l, float2* y, const float2* x, const float2* b, int nb, Gate g, cudaStream_t s) {
    BatchWS& B = *H.bws;
    const Level<float>& L = H.L32[l];
    launch_bstencil_mma(y, x, b, L.n, B.Af[l], L.Nx, L.Nt, nb, B.fp16 == 1, g, s);
}

void bapply(Handle& H, int l, float2* y, const float2* x, const float2* b, int nb, Gate g, cudaStream_t s) {
    if (l == 0) {
        const Level<float>& L = H.L32[0];
        launch_bwilson<float>(y, x, L.U, b, L.m0, L.Nx, L.Nt, L.n, nb, g, s);
    } else {
        bapply_mma(H, l, y, x, b, nb, g, s);
    }
}

// GMRES(steps) from zero on grid l for every right-hand side with an open gate
// `act`: x = V d (or x += V d), r_out = V rho (batched smoother).
void bsmoother(Handle& H, int l, const float2* f, float2* x, bool accumulate, float2* r_out, int nb, Gate act,
               cudaStream_t s) {
    BatchWS& B = *H.bws;
    BatchWS::BL& W = B.L[l];
    const long n = H.L32[l].n;
    const long row = (long)nb * n;
    double* t = B.sc + SC_LVL;
    launch_bnorm2<float>(t, NSC, f, n, n, nb, B.red, act, s);
    bks_start(W.ks, nb, t, NSC, 0.0, t, NSC, act, s);
    launch_bscale<float>(W.sV, n, f, n, MG_DEVF(W.ks, double, scale), KS_DBLS, n, nb, scale_gate(W.ks, 0), s);
    for (int jh = 0; jh < H.p.smooth_steps; ++jh)
        barnoldi_step<float>(B, [&](float2* w, const float2* in, Gate g) { bapply(H, l, w, in, nullptr, nb, g, s); },
                             W.sV, n, nb, W.ks, jh, s);
    bks_finish(W.ks, nb, s);
    launch_baxpy<float>(x, n, W.sV, row, n, 0, MG_DEVF(W.ks, int, j), KS_INTS, MG_DEVF(W.ks, double2, d), KS_CPLX,
                        1.0, !accumulate, n, nb, nullptr, 0, B.red, act, s);
    if (r_out)
        launch_baxpy<float>(r_out, n, W.sV, row, n, 1, MG_DEVF(W.ks, int, j), KS_INTS, MG_DEVF(W.ks, double2, rho),
                            KS_CPLX, 1.0, true, n, nb, nullptr, 0, B.red, act, s);
}

// GMRES-Proj(m,k) on the coarsest grid for every right-hand side with an open
// gate: projection onto the shared deflation space, then one GMRES(m - k)
// cycle, repeated (Section 2).  Counts of steps accumulate in citers.
mg_status bcoarse_proj(Handle& H, const float2* f, float2* x, int nb, Gate act, double tol, cudaStream_t s) {
    BatchWS& B = *H.bws;
    const long n = H.L32[2].n;
    const int k = H.defl_k;
    const int ms = std::max(H.p.dr_m - k, 1);
    if (ms > MSMAX || k + 1 > RED_MAXD)
        return set_error("coarse block solve: unsupported (m - k, k) = (%d, %d)", ms, k), MG_EINVAL;
    if (f != B.f2 || x != B.x2) return set_error("coarse block solve: unexpected buffers"), MG_EINVAL;
    const float2* W = H.c32.W;
    const bool fp16 = B.fp16 == 1;
    k_gate_to_flags<<<(nb + 63) / 64, 64, 0, s>>>(B.cact, act, nb);
    count_launch();
    const Gate ca{B.cact, 1, 1};
    double* cnb2 = B.sc + SC_CNB2;
    double* cr2 = B.sc + SC_CR2;
    launch_bnorm2<float>(cnb2, NSC, f, n, n, nb, B.red, ca, s);
    MG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)nb * n * sizeof(float2), s));
    MG_CUDA_TRY(cudaMemcpyAsync(B.cr, f, (size_t)nb * n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MG_CUDA_TRY(cudaMemsetAsync(B.ccycles, 0, sizeof(int), s));
    const long row = (long)nb * n;
    CBArgs cb{};
    cb.Af = B.Af[2];
    cb.Nx = H.L32[2].Nx;
    cb.Nt = H.L32[2].Nt;
    cb.n = n;
    cb.V = B.cV;
    cb.row = row;
    cb.ks = B.cks;
    cb.gbuf = B.cgb;
    cb.p1 = B.cp1;
    cb.p2 = B.cp2;
    cb.h1 = B.ch1;
    cb.h2 = B.ch2;
    cb.ticket = B.ctk;
    cb.bar = B.cbar;
    cb.probe = B.probe;
    // the cycle kernel when its grid can be resident at once, else the step kernels
    const bool coop = !B.no_coop && cb_geometry_cycle(cb, (long)cb.Nx * cb.Nt, nb, fp16);
    if (!coop) cb_geometry(cb, (long)cb.Nx * cb.Nt, nb);
    const long spin = B.spin > 0 ? B.spin : 1L << 18;  // polls of a tile barrier before it gives up
    if (B.probe && !coop) return set_error("the coarse timeout probe is built into the cycle kernel only"), MG_EINVAL;
    if ((long)nb * CB_PB * CB_MAXCH > B.cp_cap || cb.nchunks > CB_MAXCH || (!coop && cb.spc > CB_MAXSPC))
        return set_error("coarse block solve: %d coarse sites exceed the fused step's chunking", cb.Nx * cb.Nt), MG_EINVAL;
    // one cycle: projection d = argmin ||W^+ r - H_k d||, x += W_k d, r -= W H_k d,
    // then one GMRES(ms) cycle from r, x += V d, r = V rho; every kernel gated per
    // right-hand side, so the same sequence serves every cycle
    auto cycle = [&](cudaStream_t cs) {
        launch_bgram<float>(B.cg, KLD, W, n, 0, k + 1, nullptr, 0, B.cr, n, n, nb, B.red, ca, cs);
        bproj_solve(H.pls, nb, B.cg, KLD, B.cd, KLD, B.cu, KLD, ca, cs);
        launch_baxpy<float>(x, n, W, n, 0, k, nullptr, 0, B.cd, KLD, 1.0, false, n, nb, nullptr, 0, B.red, ca, cs);
        launch_baxpy<float>(B.cr, n, W, n, 0, k + 1, nullptr, 0, B.cu, KLD, -1.0, false, n, nb, cr2, NSC, B.red, ca,
                            cs);
        bks_start(B.cks, nb, cr2, NSC, tol, cnb2, NSC, ca, cs);
        launch_cb_gate_init(cb, cs);
        launch_bscale<float>(B.cV, n, B.cr, n, MG_DEVF(B.cks, double, scale), KS_DBLS, n, nb, scale_gate(B.cks, 0),
                             cs);
        if (coop) (void)launch_cb_cycle(cb, ms, fp16, spin, B.count + 1, cs);
        else
            for (int jh = 0; jh < ms; ++jh) launch_cb_step(cb, jh, fp16, cs);
        bks_finish(B.cks, nb, cs);
        launch_baxpy<float>(x, n, B.cV, row, n, 0, MG_DEVF(B.cks, int, j), KS_INTS, MG_DEVF(B.cks, double2, d),
                            KS_CPLX, 1.0, false, n, nb, nullptr, 0, B.red, ca, cs);
        launch_baxpy<float>(B.cr, n, B.cV, row, n, 1, MG_DEVF(B.cks, int, j), KS_INTS, MG_DEVF(B.cks, double2, rho),
                            KS_CPLX, 1.0, true, n, nb, nullptr, 0, B.red, ca, cs);
        k_coarse_cycle_end<<<1, 64, 0, cs>>>(B.cact, B.citers, B.cks, nb, B.ccycles, H.p.proj_max_cycles, B.count);
        count_launch();
    };
    // the cycle as a CUDA graph, captured once per (block size, deflation size, tolerance, format)
    if (!B.cyc_exec || B.cyc_nb != nb || B.cyc_k != k || B.cyc_tol != tol || B.cyc_fp16 != (fp16 ? 1 : 0) ||
        B.cyc_coop != (coop ? 1 : 0) || B.cyc_probe != B.probe || B.cyc_spin != spin) {
        if (B.cyc_exec) cudaGraphExecDestroy(B.cyc_exec);
        B.cyc_exec = nullptr;
        if (!B.cap) MG_CUDA_TRY(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
        const unsigned long long before = g_launches.load();
        MG_CUDA_TRY(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
        cycle(B.cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(B.cap, &g);
        const unsigned long long kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);  // counted per replay instead
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = (ce == cudaSuccess) ? cudaGraphInstantiate(&ex, g, 0) : ce;
        if (g) cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            (void)cudaGetLastError();
            if (coop) {  // capture the step kernels instead
                B.no_coop = true;
                return bcoarse_proj(H, f, x, nb, act, tol, s);
            }
            return set_error("coarse cycle graph: %s", cudaGetErrorString(ie)), MG_ECUDA;
        }
        B.cyc_exec = ex;
        B.cyc_nb = nb;
        B.cyc_k = k;
        B.cyc_tol = tol;
        B.cyc_fp16 = fp16 ? 1 : 0;
        B.cyc_coop = coop ? 1 : 0;
        B.cyc_probe = B.probe;
        B.cyc_spin = spin;
        B.cyc_kernels = kernels;
    }
    for (int i = 0; i < 2; ++i)
        if (!B.ev[i]) MG_CUDA_TRY(cudaEventCreateWithFlags(&B.ev[i], cudaEventDisableTiming));
    // cycles replay back to back; the host reads the active count of cycle c while
    // cycle c + 1 runs (a cycle with every right-hand side stopped changes nothing)
    int* hc = reinterpret_cast<int*>(static_cast<char*>(B.pin) + 40960);
    auto launch_cycle = [&](int c) -> mg_status {
        MG_CUDA_TRY(cudaGraphLaunch(B.cyc_exec, s));
        count_launch(B.cyc_kernels);
        MG_CUDA_TRY(cudaMemcpyAsync(hc + 2 * (c & 1), B.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        MG_CUDA_TRY(cudaEventRecord(B.ev[c & 1], s));
        return MG_OK;
    };
    MG_TRY(launch_cycle(0));
    bool gave_up = false;
    for (int c = 0; c <= H.p.proj_max_cycles; ++c) {
        MG_TRY(launch_cycle(c + 1));
        MG_CUDA_TRY(cudaEventSynchronize(B.ev[c & 1]));
        gave_up = gave_up || hc[2 * (c & 1) + 1] != 0;
        if (hc[2 * (c & 1)] == 0 || gave_up) break;
    }
    if (gave_up) {
        // every launch has ended (each wait is bounded); the barrier counts may be
        // left mid-count, so they restart from zero with the error flag
        MG_CUDA_TRY(cudaStreamSynchronize(s));
        MG_CUDA_TRY(cudaMemsetAsync(B.count + 1, 0, sizeof(int), s));
        MG_CUDA_TRY(cudaMemsetAsync(B.cbar, 0, (2 * NB_MAX / NB_TILE + 1) * sizeof(unsigned), s));
        return set_error("coarse block solve: a tile barrier gave up"), MG_ETIMEOUT;
    }
    return MG_OK;
}

// the batched V-cycle of grid 0 for the right-hand sides with an open gate:
// x = S(f); x += P (grid 1 cycle on P^+ r); r = f - A x; x += S(r), and on grid 1
// the same with the coarsest solve in place of the grid-2 cycle
mg_status bvcycle(Handle& H, const float2* f, float2* x, int nb, Gate act, cudaStream_t s) {
    BatchWS& B = *H.bws;
    Level<float>* Ls = H.L32;
    const long n0 = Ls[0].n, n1 = Ls[1].n, n2 = Ls[2].n;
    bsmoother(H, 0, f, x, false, B.L[0].r, nb, act, s);
    launch_brestrict<float>(B.L[1].f, n1, B.L[0].r, n0, Ls[0].Q, Ls[0].Nx, Ls[0].Nt, Ls[0].h, nb, act, s);
    bsmoother(H, 1, B.L[1].f, B.L[1].x, false, B.L[1].r, nb, act, s);
    launch_brestrict<float>(B.f2, n2, B.L[1].r, n1, Ls[1].Q, Ls[1].Nx, Ls[1].Nt, Ls[1].h, nb, act, s);
    MG_TRY(bcoarse_proj(H, B.f2, B.x2, nb, act, H.p.coarse_tol_rest, s));
    launch_bprolong<float>(B.L[1].x, n1, B.x2, n2, Ls[1].Q, Ls[1].Nx, Ls[1].Nt, Ls[1].h, true, nb, act, s);
    bapply(H, 1, B.L[1].r, B.L[1].x, B.L[1].f, nb, act, s);  // r = f - A x
    bsmoother(H, 1, B.L[1].r, B.L[1].x, true, nullptr, nb, act, s);
    launch_bprolong<float>(x, n0, B.L[1].x, n1, Ls[0].Q, Ls[0].Nx, Ls[0].Nt, Ls[0].h, true, nb, act, s);
    bapply(H, 0, B.L[0].r, x, f, nb, act, s);
    bsmoother(H, 0, B.L[0].r, x, true, nullptr, nb, act, s);
    return MG_OK;
}

}  // namespace

// FGMRES(m) in FP64 for nb right-hand sides in lockstep (device B, X: [nb][n0]),
// each with its own Krylov space and convergence on its own true residual.
mg_status fgmres_solve_block(Handle& H, const double2* Bv, double2* X, int nb, double tol, bool fp16, cudaStream_t s,
                             int* iters, double* relres, bool* converged, long long* coarse_iters) {
    const int nbp = ((nb + NB_TILE - 1) / NB_TILE) * NB_TILE;
    MG_TRY(batch_alloc(H, nbp, fp16, s));
    BatchWS& B = *H.bws;
    const Level<double>& L0 = H.L64[0];
    const long n0 = L0.n;
    const int m = H.p.fgmres_m;
    const long row = (long)nbp * n0;
    // padded right-hand sides are zero (closed from the start); b may be host or device memory
    MG_CUDA_TRY(cudaMemsetAsync(B.fb, 0, (size_t)nbp * n0 * sizeof(double2), s));
    MG_CUDA_TRY(cudaMemcpyAsync(B.fb, Bv, (size_t)nb * n0 * sizeof(double2), cudaMemcpyDefault, s));
    MG_CUDA_TRY(cudaMemsetAsync(B.fx, 0, (size_t)nbp * n0 * sizeof(double2), s));
    MG_CUDA_TRY(cudaMemsetAsync(B.citers, 0, (size_t)nbp * sizeof(long long), s));
    double* fnb2 = B.sc + SC_FNB2;
    double* r2 = B.sc + SC_R2;
    launch_bnorm2<double>(fnb2, NSC, B.fb, n0, n0, nbp, B.red, Gate{}, s);
    MG_CUDA_TRY(cudaMemcpyAsync(B.fr, B.fb, (size_t)nbp * n0 * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    std::vector<double> nbv(nbp), r2v(nbp);
    double* hsc = static_cast<double*>(B.pin);
    MG_CUDA_TRY(cudaMemcpyAsync(hsc, B.sc, (size_t)nbp * NSC * sizeof(double), cudaMemcpyDeviceToHost, s));
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> act(nbp, 0), outer(nbp, 0);
    for (int r = 0; r < nbp; ++r) {
        nbv[r] = std::sqrt(hsc[r * NSC + SC_FNB2]);
        act[r] = (r < nb && nbv[r] > 0.0) ? 1 : 0;
        if (r < nb) {
            iters[r] = 0;
            relres[r] = 0.0;
            converged[r] = !act[r];
        }
    }
    int* dflags = B.oflags;
    auto any_active = [&]() {
        for (int r = 0; r < nbp; ++r)
            if (act[r]) return true;
        return false;
    };
    const Gate oa{dflags, 1, 1};
    long long true_residuals = 0;
    while (any_active()) {
        int* hf = reinterpret_cast<int*>(static_cast<char*>(B.pin) + 32768);
        std::memcpy(hf, act.data(), (size_t)nbp * sizeof(int));
        MG_CUDA_TRY(cudaMemcpyAsync(dflags, hf, (size_t)nbp * sizeof(int), cudaMemcpyHostToDevice, s));
        launch_bnorm2<double>(r2, NSC, B.fr, n0, n0, nbp, B.red, oa, s);
        bks_start(B.fks, nbp, r2, NSC, tol, fnb2, NSC, oa, s);
        launch_bscale<double>(B.fV, n0, B.fr, n0, MG_DEVF(B.fks, double, scale), KS_DBLS, n0, nbp,
                              scale_gate(B.fks, 0), s);
        std::vector<int> cyc(act);  // right-hand sides still stepping in this cycle
        for (int jh = 0; jh < m; ++jh) {
            const Gate sg = step_gate(B.fks, jh);
            launch_bconvert<double, float>(B.v32, n0, B.fV + (long)jh * row, n0, n0, nbp, s);
            MG_TRY(bvcycle(H, B.v32, B.z32, nbp, sg, s));
            launch_bconvert<float, double>(B.fZ + (long)jh * row, n0, B.z32, n0, n0, nbp, s);
            const double2* zj = B.fZ + (long)jh * row;
            barnoldi_step<double>(
                B,
                [&](double2* w, const double2*, Gate g) {
                    launch_bwilson<double>(w, zj, L0.U, nullptr, L0.m0, L0.Nx, L0.Nt, n0, nbp, g, s);
                },
                B.fV, n0, nbp, B.fks, jh, s);
            // host: which right-hand sides continue (one small read per outer step)
            k_gather_gates<<<(nbp + 63) / 64, 64, 0, s>>>(B.gates, B.fks, nbp);
            count_launch();
            int* gates = static_cast<int*>(B.pin);
            MG_CUDA_TRY(cudaMemcpyAsync(gates, B.gates, (size_t)nbp * sizeof(int), cudaMemcpyDeviceToHost, s));
            MG_CUDA_TRY(cudaStreamSynchronize(s));
            bool more = false;
            for (int r = 0; r < nbp; ++r) {
                if (!cyc[r]) continue;
                ++outer[r];
                cyc[r] = gates[r] == jh + 1 ? 1 : 0;
                more = more || cyc[r];
            }
            if (!more) break;
        }
        bks_finish(B.fks, nbp, s);
        launch_baxpy<double>(B.fx, n0, B.fZ, row, n0, 0, MG_DEVF(B.fks, int, j), KS_INTS, MG_DEVF(B.fks, double2, d),
                             KS_CPLX, 1.0, false, n0, nbp, nullptr, 0, B.red, oa, s);
        launch_bwilson<double>(B.fr, B.fx, L0.U, B.fb, L0.m0, L0.Nx, L0.Nt, n0, nbp, oa, s);  // true residual
        for (int r = 0; r < nb; ++r) true_residuals += act[r];
        launch_bnorm2<double>(r2, NSC, B.fr, n0, n0, nbp, B.red, oa, s);
        MG_CUDA_TRY(cudaMemcpyAsync(hsc, B.sc, (size_t)nbp * NSC * sizeof(double), cudaMemcpyDeviceToHost, s));
        MG_CUDA_TRY(cudaStreamSynchronize(s));
        for (int r = 0; r < nb; ++r) {
            if (!act[r]) continue;
            relres[r] = std::sqrt(hsc[r * NSC + SC_R2]) / nbv[r];
            if (relres[r] <= tol) {
                converged[r] = true;
                act[r] = 0;
            } else if (outer[r] >= H.p.max_outer) {
                act[r] = 0;
            }
        }
    }
    for (int r = 0; r < nb; ++r) iters[r] = outer[r];
    MG_CUDA_TRY(cudaMemcpyAsync(X, B.fx, (size_t)nb * n0 * sizeof(double2), cudaMemcpyDefault, s));
    std::vector<long long> ci(nbp);
    MG_CUDA_TRY(cudaMemcpyAsync(B.pin, B.citers, (size_t)nbp * sizeof(long long), cudaMemcpyDeviceToHost, s));
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(ci.data(), B.pin, (size_t)nbp * sizeof(long long));
    long long tot = 0;
    for (int r = 0; r < nb; ++r) tot += ci[r];
    if (coarse_iters) *coarse_iters = tot;
    H.st.coarse_iters += tot;
    H.st.mvps[2] += tot;
    int sum_outer = 0;
    for (int r = 0; r < nb; ++r) sum_outer += outer[r];
    H.st.outer += sum_outer;
    // operator applications per outer step: on the fine grid two smoothers, the
    // residual and the FP64 Arnoldi apply; on the intermediate grid two smoothers
    // and the residual; one coarse solve.  Plus one FP64 true residual per cycle.
    H.st.mvps[0] += (long long)sum_outer * (2 * H.p.smooth_steps + 2) + true_residuals;
    H.st.mvps[1] += (long long)sum_outer * (2 * H.p.smooth_steps + 1);
    H.st.coarse_solves += sum_outer;
    return MG_OK;
}

// batched coarse GMRES-Proj alone (the C ABI's parity entry): device f, x [nb][n2]
mg_status coarse_solve_block(Handle& H, const float2* f, float2* x, int nb, double tol, bool fp16, cudaStream_t s,
                             long long* iters, bool probe, long spin) {
    const int nbp = ((nb + NB_TILE - 1) / NB_TILE) * NB_TILE;
    MG_TRY(batch_alloc(H, nbp, fp16, s));
    BatchWS& B = *H.bws;
    const long n2 = H.L32[2].n;
    MG_CUDA_TRY(cudaMemsetAsync(B.f2, 0, (size_t)nbp * n2 * sizeof(float2), s));
    MG_CUDA_TRY(cudaMemcpyAsync(B.f2, f, (size_t)nb * n2 * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MG_CUDA_TRY(cudaMemsetAsync(B.citers, 0, (size_t)nbp * sizeof(long long), s));
    int* hf = static_cast<int*>(B.pin);
    for (int r = 0; r < nbp; ++r) hf[r] = r < nb ? 1 : 0;
    int* dflags = B.oflags;
    MG_CUDA_TRY(cudaMemcpyAsync(dflags, hf, (size_t)nbp * sizeof(int), cudaMemcpyHostToDevice, s));
    B.probe = probe ? 1 : 0;
    B.spin = spin;
    const mg_status st = bcoarse_proj(H, B.f2, B.x2, nbp, Gate{dflags, 1, 1}, tol, s);
    B.probe = 0;
    B.spin = 0;
    if (st != MG_OK && st != MG_ETIMEOUT) return st;
    MG_CUDA_TRY(cudaMemcpyAsync(x, B.x2, (size_t)nb * n2 * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MG_CUDA_TRY(cudaMemcpyAsync(B.pin, B.citers, (size_t)nbp * sizeof(long long), cudaMemcpyDeviceToHost, s));
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    if (iters) std::memcpy(iters, B.pin, (size_t)nb * sizeof(long long));
    return st;
}

// block stencil apply alone (parity entry): device x, y [nb][n_l] complex64, grid l = 1, 2
mg_status apply_block(Handle& H, int l, const float2* x, float2* y, int nb, bool fp16, cudaStream_t s) {
    if (nb % NB_TILE) return set_error("the block apply takes a multiple of %d right-hand sides", NB_TILE), MG_EINVAL;
    MG_TRY(batch_alloc(H, nb, fp16, s));
    bapply_mma(H, l, y, x, nullptr, nb, Gate{}, s);
    MG_LAUNCH_CHECK();
    return MG_OK;
}

}  // namespace mg
