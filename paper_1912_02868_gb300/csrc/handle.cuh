// The hierarchy handle: device buffers of all three grids in FP64 and FP32,
// Krylov workspaces, the coarse deflation space, and host-side counters.
#pragma once
#include <vector>

#include "coarse_coop.cuh"
#include "kstate.cuh"
#include "setup.cuh"

struct mg_handle_s;

namespace mg {

struct BatchWS;                  // workspaces of the lockstep block solve (solver_batch.cu)
void destroy_batch(BatchWS* B);

// CUDA-event timing of every operator apply on one grid (for roofline reports).
struct ApplyTimer {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // start/stop pairs, reused
    size_t used = 0;
    cudaEvent_t next() {
        if (used == ev.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev.push_back(e);
        }
        return ev[used++];
    }
};

// One grid of the hierarchy in one precision.
template <typename T>
struct Level {
    int Nx = 0, Nt = 0, dof = 0;
    long n = 0;                   // complex entries of a vector
    const C2<T>* U = nullptr;     // level 0: gauge field
    double m0 = 0.0;
    const C2<T>* A = nullptr;     // levels 1, 2: stencil (column-major blocks)
    const C2<T>* F = nullptr;     // level 1 with lowrank_hops: the stencil with rank-4 hop factors
    const C2<T>* Q = nullptr;     // prolongator to the next grid (none on the coarsest)
    int h = 1;                    // dofs per chirality at this grid
    // workspaces
    C2<T>* sV = nullptr;          // smoother basis, (smooth_steps + 1) x n
    C2<T>* x = nullptr;           // cycle output
    C2<T>* f = nullptr;           // cycle input (levels 1, 2)
    C2<T>* r = nullptr;           // residual
    KState* ks = nullptr;         // smoother state
    ApplyTimer* timer = nullptr;  // shared by both precisions of the grid
    int shape = 0;                // launch shape of the apply (0: built-in; tune.cu)
    double shape_us[2] = {0, 0};  // the tuner's times of the chosen and the built-in shape

    void apply(C2<T>* y, const C2<T>* xin, const C2<T>* b, bool dagger, Gate g, cudaStream_t s) const {
        cudaEvent_t e1 = nullptr;
        if (timer && timer->on) {
            cudaEvent_t e0 = timer->next();
            e1 = timer->next();
            if (e0) cudaEventRecord(e0, s);
        }
        if (U) launch_wilson<T>(y, xin, U, b, m0, Nx, Nt, dagger, g, s, shape);
        else if (F) launch_stencil_lr<T>(y, xin, F, b, Nx, Nt, dagger, g, s, shape);
        else launch_stencil<T>(y, xin, A, b, Nx, Nt, dof, dagger, g, s, shape);
        if (e1) cudaEventRecord(e1, s);
    }
};

// Coarsest-grid Krylov workspace in one precision.
template <typename T>
struct CoarseWS {
    C2<T>* V = nullptr;   // (dr_m + 1) x n2
    C2<T>* V2 = nullptr;  // restart target, (dr_m + 1) x n2
    C2<T>* r = nullptr;
    C2<T>* p = nullptr;   // CG
    C2<T>* q = nullptr;
    C2<T>* t = nullptr;
    C2<T>* W = nullptr;   // deflation space rows (dr_k + 1) x n2
    KState* ks = nullptr;
};

// Intermediate-grid FGMRES of the partial solve (mg_params.partial_tol > 0), one precision.
template <typename T>
struct PartialWS {
    C2<T>* V = nullptr;   // (fgmres_m + 1) x n1
    C2<T>* Z = nullptr;   // fgmres_m x n1
    C2<T>* r = nullptr;
    KState* ks = nullptr;
};

struct Scalars {  // device scalars of the host-driven loops
    double nb2;       // ||b||^2 of the current solve
    double r2;        // ||r||^2
    double tmp[8];
    double rr, pq, rr_new;
    int cg_active, cg_iters;
    int err;
};

struct Stats {
    long long mvps[3] = {0, 0, 0};
    int outer = 0;
    int coarse_solves = 0;
    long long coarse_iters = 0;
    int dr_solves = 0;
};

// The captured mixed V-cycle of a handle (mg_params.vcycle_graph): the graph,
// the deflation size it was captured with, its kernel count and the counters
// one replay adds.
struct VGraph {
    cudaGraphExec_t exec = nullptr;
    int k = 0;
    unsigned long long kernels = 0;
    Stats per_replay;
    int eligible_runs = 0;  // eligible V-cycles run before capture (the first warms the launch set-up)
};

struct Handle {
    int Lx = 0, Lt = 0;
    double m0 = 0.0;
    mg_params p{};
    std::vector<void*> allocs;
    void* pinned = nullptr;       // host staging for status reads
    RedWS red;
    Scalars* sc = nullptr;
    Level<double> L64[3];
    Level<float> L32[3];
    // device copies of the set-up in FP64 (owned; the Level views point into them)
    double2* U64 = nullptr;
    double2* A64[3] = {nullptr, nullptr, nullptr};
    double2* Q64[2] = {nullptr, nullptr};
    float2* U32 = nullptr;
    float2* A32[3] = {nullptr, nullptr, nullptr};
    unsigned* A16c = nullptr;  // FP16 copy of the coarsest operator for the cluster kernels (coarse_half)
    double2* F64 = nullptr;    // intermediate grid with rank-4 hop factors (lowrank_hops), LR_SITE per site
    float2* F32 = nullptr;
    double lowrank_err = 0.0;  // largest relative error of the factored hop blocks
    float2* Q32[2] = {nullptr, nullptr};
    // fine FGMRES (FP64)
    double2* fV = nullptr;  // (m+1) x n0
    double2* fZ = nullptr;  // m x n0
    double2* fx = nullptr;
    double2* fr = nullptr;
    double2* fb = nullptr;
    float2* v32 = nullptr;
    float2* z32 = nullptr;
    KState* fks = nullptr;
    // coarsest grid
    CoarseWS<double> c64;
    CoarseWS<float> c32;
    double2* cvec = nullptr;  // (k+1) Gram coefficients of a projection
    double2* dvec = nullptr;
    double2* uvec = nullptr;
    DRState* dr = nullptr;
    KState* pls = nullptr;    // factored H_k of the deflation space
    double2* cpart = nullptr; // partial sums of the cooperative coarse solve
    int cpart_ctas = 0;
    CoopStats* cstats = nullptr;
    // fine-grid deflation arm (method MG_METHOD_FINE_DEFLATION), FP64
    double2* fdV = nullptr;   // (m+1) x n0
    double2* fdV2 = nullptr;
    double2* fcg[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // fine CGNE: y, r, p, q, t
    double2* fdW = nullptr;   // (k+1) x n0
    KState* fdks = nullptr;
    KState* fdpls = nullptr;
    int fine_k = 0;
    // partial intermediate solve
    PartialWS<double> p64;
    PartialWS<float> p32;
    int cur_outer = 0;        // outer FGMRES step being preconditioned (picks the coarse tolerance)
    int defl_k = 0;           // 0: no deflation space yet
    Stats st;
    ApplyTimer timers[3];
    // concurrent solve contexts sharing this hierarchy (mg_solve with nrhs > 1)
    bool is_context = false;             // a context: shares hierarchy and deflation, owns workspaces
    cudaStream_t own_stream = nullptr;   // a context's stream
    cudaStream_t work_stream = nullptr;  // this handle's stream for its share of a parallel solve
    cudaStream_t cap_stream = nullptr;   // stream the V-cycle graph is captured on
    VGraph vg;
    std::vector<mg_handle_s*> contexts;
    size_t bytes = 0;                    // device bytes this handle allocated
    BatchWS* bws = nullptr;              // block-solve workspaces (allocated by the first block solve)

    template <typename T> Level<T>* levels();
    template <typename T> CoarseWS<T>& coarse();
    template <typename T> PartialWS<T>& partial();
};
template <> inline Level<double>* Handle::levels<double>() { return L64; }
template <> inline Level<float>* Handle::levels<float>() { return L32; }
template <> inline CoarseWS<double>& Handle::coarse<double>() { return c64; }
template <> inline CoarseWS<float>& Handle::coarse<float>() { return c32; }
template <> inline PartialWS<double>& Handle::partial<double>() { return p64; }
template <> inline PartialWS<float>& Handle::partial<float>() { return p32; }

// allocation owned by the handle
mg_status halloc(Handle& H, void** p, size_t bytes);
template <typename P> mg_status halloc_t(Handle& H, P** p, size_t count) {
    return halloc(H, reinterpret_cast<void**>(p), count * sizeof(P));
}

// solve entry points (solver.cu)
mg_status fgmres_solve(Handle& H, const double2* b, double2* x, double tol, cudaStream_t s, int* iters,
                       double* relres, bool* converged);
// Two right-hand sides on two contexts of one hierarchy, in lockstep with paired
// coarsest solves (mixed precision, deflation space built); solver.cu.
mg_status fgmres_solve_pair(Handle* HH[2], const double2* const b[2], double2* const x[2], double tol,
                            cudaStream_t s, int it_out[2], double rr_out[2], bool conv_out[2]);
mg_status build_hierarchy(Handle& H, const double2* gauge_dev, const double2* starts0, const double2* starts1,
                          const double2* nullvecs0, const double2* nullvecs1, cudaStream_t s);
mg_status fine_cgne_solve(Handle& H, const double2* b, double2* x, double tol, cudaStream_t s, int* iters,
                          double* relres, bool* converged);
mg_status fine_deflated_solve(Handle& H, const double2* b, double2* x, double tol, cudaStream_t s, int* iters,
                              double* relres, bool* converged);
// Lockstep FGMRES of nb <= 64 right-hand sides (host or device b, x: [nb][n0]) with
// the batched V-cycle and tensor-core block products (solver_batch.cu); needs the
// deflation space.  coarse_iters (optional): coarse GMRES-Proj steps of the block.
mg_status fgmres_solve_block(Handle& H, const double2* B, double2* X, int nb, double tol, bool fp16, cudaStream_t s,
                             int* iters, double* relres, bool* converged, long long* coarse_iters);
// the batched coarse GMRES-Proj alone (device f, x: [nb][n2] complex64); probe: every
// CTA of the cycle kernel first waits on a word nothing writes, giving up after
// `spin` polls (spin 0: the default limit); MG_ETIMEOUT when a wait gave up
mg_status coarse_solve_block(Handle& H, const float2* f, float2* x, int nb, double tol, bool fp16, cudaStream_t s,
                             long long* iters, bool probe = false, long spin = 0);
// the tensor-core block stencil of grid l alone (device x, y: [nb][n_l] complex64, nb % 8 == 0)
mg_status apply_block(Handle& H, int l, const float2* x, float2* y, int nb, bool fp16, cudaStream_t s);
// Launch shapes of the handle's level applies chosen by timing (tune.cu), at set-up
mg_status tune_shapes(Handle& H, cudaStream_t s);
// A solve context of `owner` (capi.cu): same hierarchy and deflation space,
// own workspaces and stream; usable with mg_solve and released with mg_destroy
// (before its owner).  The owner's deflation space must exist.
mg_status make_solve_context(mg_handle_s* owner, mg_handle_s** out);
size_t handle_device_bytes(const mg_handle_s* h);
cudaStream_t handle_stream(const mg_handle_s* h);

}  // namespace mg

struct mg_handle_s {
    mg::Handle h;
};
