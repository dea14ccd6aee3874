// Launch-shape autotuner (mg_params.autotune).
//
// The level applies -- the fine Wilson-Dirac apply and the FP32 block stencils
// of the intermediate and coarsest grids -- take a launch shape that only groups
// sites into blocks (threads per block for the one-thread-per-site Wilson
// kernel, 32 x r tiles for the shared-memory one, sites a lane for the
// register-column one; sites per block for the stencils).  Each site's arithmetic, and so
// every result bit, is the same for all shapes; only the speed differs.  At
// set-up, every tunable apply of the handle is timed with each candidate shape
// and with the built-in one, on the handle's stream and its own workspace
// vectors, and the fastest is kept.  A candidate replaces the built-in shape
// only when it is at least 3% faster, so timing noise does not flip choices
// that make no difference.  Choices are cached per (device, kernel, precision,
// grid size) for the process: handles of one size tune once.
#include <mutex>
#include <vector>

#include "handle.cuh"

namespace mg {

namespace {

enum TuneKind { TK_WILSON = 0, TK_STENCIL_LR = 1, TK_STENCIL = 2 };

struct TuneEntry {
    int dev, kind, prec;
    long nsite;
    int shape;
    double us[2];  // chosen, built-in
};

std::mutex tune_mu;
std::vector<TuneEntry> tune_cache;

constexpr int TUNE_WARM = 3;
constexpr int TUNE_REPS = 10;
constexpr double TUNE_MARGIN = 0.97;

// mean time of one apply of L with launch shape `shape` (microseconds)
template <typename T>
mg_status time_apply(Level<T>& L, int shape, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* us) {
    const int saved = L.shape;
    ApplyTimer* const tm = L.timer;
    L.shape = shape;
    L.timer = nullptr;  // no per-apply events while tuning
    const Gate open{};
    for (int i = 0; i < TUNE_WARM; ++i) L.apply(L.x, L.r, nullptr, false, open, s);
    MG_CUDA_TRY(cudaEventRecord(e0, s));
    for (int i = 0; i < TUNE_REPS; ++i) L.apply(L.x, L.r, nullptr, false, open, s);
    MG_CUDA_TRY(cudaEventRecord(e1, s));
    L.shape = saved;
    L.timer = tm;
    MG_CUDA_TRY(cudaGetLastError());
    MG_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    MG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *us = 1e3 * (double)ms / TUNE_REPS;
    return MG_OK;
}

template <typename T>
mg_status tune_level(Level<T>& L, int dev, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    if (!L.x || !L.r || L.n <= 0) return MG_OK;
    const bool f32 = std::is_same<T, float>::value;
    int kind;
    const int* cand;
    int ncand;
    if (L.U) {
        kind = TK_WILSON;
        cand = WILSON_SHAPES;
        ncand = (int)(sizeof(WILSON_SHAPES) / sizeof(int));
    } else if (!f32) {
        return MG_OK;  // the FP64 stencils have one shape
    } else if (L.F) {
        kind = TK_STENCIL_LR;
        cand = STENCIL_LR_F32_SHAPES;
        ncand = (int)(sizeof(STENCIL_LR_F32_SHAPES) / sizeof(int));
    } else if (L.A) {
        kind = TK_STENCIL;
        cand = STENCIL_F32_SHAPES;
        ncand = (int)(sizeof(STENCIL_F32_SHAPES) / sizeof(int));
    } else {
        return MG_OK;
    }
    const long nsite = (long)L.Nx * L.Nt;
    const int prec = f32 ? 1 : 0;
    {
        std::lock_guard<std::mutex> lock(tune_mu);
        for (const TuneEntry& e : tune_cache)
            if (e.dev == dev && e.kind == kind && e.prec == prec && e.nsite == nsite) {
                L.shape = e.shape;
                L.shape_us[0] = e.us[0];
                L.shape_us[1] = e.us[1];
                return MG_OK;
            }
    }
    MG_CUDA_TRY(cudaMemsetAsync(L.r, 0, sizeof(C2<T>) * (size_t)L.n, s));
    double t0 = 0.0;
    MG_TRY(time_apply(L, 0, s, e0, e1, &t0));
    int best = 0;
    double tb = t0;
    for (int i = 0; i < ncand; ++i) {
        double t = 0.0;
        MG_TRY(time_apply(L, cand[i], s, e0, e1, &t));
        if (t < tb) {
            tb = t;
            best = cand[i];
        }
    }
    if (best != 0 && tb > TUNE_MARGIN * t0) {
        best = 0;
        tb = t0;
    }
    L.shape = best;
    L.shape_us[0] = tb;
    L.shape_us[1] = t0;
    std::lock_guard<std::mutex> lock(tune_mu);
    tune_cache.push_back(TuneEntry{dev, kind, prec, nsite, best, {tb, t0}});
    return MG_OK;
}

}  // namespace

mg_status tune_shapes(Handle& H, cudaStream_t s) {
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MG_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return MG_ECUDA;
    }
    mg_status st = MG_OK;
    for (int l = 0; l < 3 && st == MG_OK; ++l) {
        st = tune_level(H.L64[l], dev, s, e0, e1);
        if (st == MG_OK) st = tune_level(H.L32[l], dev, s, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace mg
