// The C ABI declared in include/mg.h: argument checks, buffer management,
// host/device pointer handling, and error reporting.  No arithmetic of the
// method is done here; it only calls the kernels and the solver orchestration.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>
#include <string>
#include <memory>
#include <thread>
#include <vector>
#include <algorithm>

#include "handle.cuh"

namespace mg {

static thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int sm_count() {
    static int cache[16] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= 16) return 152;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

mg_status halloc(Handle& H, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        (void)cudaGetLastError();
        return MG_ENOMEM;
    }
    H.allocs.push_back(*p);
    H.bytes += bytes;
    return MG_OK;
}

template <typename T> mg_status vcycle_entry(Handle& H, const C2<T>* f, C2<T>* x, cudaStream_t s);

namespace {

void free_handle(Handle& H) {
    for (mg_handle_s* c : H.contexts) {
        free_handle(c->h);
        delete c;
    }
    H.contexts.clear();
    if (H.own_stream) cudaStreamDestroy(H.own_stream);
    H.own_stream = nullptr;
    if (H.work_stream) cudaStreamDestroy(H.work_stream);
    H.work_stream = nullptr;
    destroy_batch(H.bws);
    H.bws = nullptr;
    if (H.vg.exec) cudaGraphExecDestroy(H.vg.exec);
    H.vg = VGraph{};
    if (H.cap_stream) cudaStreamDestroy(H.cap_stream);
    H.cap_stream = nullptr;
    for (auto& t : H.timers) {
        for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
        t.ev.clear();
    }
    for (void* p : H.allocs) cudaFree(p);
    H.allocs.clear();
    if (H.pinned) cudaFreeHost(H.pinned);
    H.pinned = nullptr;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mg_status check_params(const mg_params& p) {
    if (p.levels != 3) return set_error("only 3 grids are built (levels = %d)", p.levels), MG_EINVAL;
    if (p.block != 4) return set_error("only 4^2 blocking is built (block = %d)", p.block), MG_EINVAL;
    if (p.nvec != 12) return set_error("only 12 near-null vectors are built (nvec = %d)", p.nvec), MG_EINVAL;
    if (p.smooth_steps < 1 || p.smooth_steps > 8) return set_error("smooth_steps must be in [1, 8]"), MG_EINVAL;
    if (p.fgmres_m < 1 || p.fgmres_m > KMAX - 1) return set_error("fgmres_m must be in [1, %d]", KMAX - 1), MG_EINVAL;
    if (p.dr_m < 2 || p.dr_m > KMAX - 1 || p.dr_m + 1 > RED_MAXD)
        return set_error("dr_m must be in [2, %d]", KMAX - 1), MG_EINVAL;
    if (p.dr_k < 1 || p.dr_k >= p.dr_m) return set_error("dr_k must be in [1, dr_m)"), MG_EINVAL;
    if (p.max_outer < 1 || p.dr_max_cycles < 1 || p.proj_max_cycles < 1 || p.cgne_max_iters < 1 ||
        p.nullvec_max_iters < 1 || p.dr_stall_cycles < 1)
        return set_error("iteration limits must be positive"), MG_EINVAL;
    if (!(p.nullvec_tol > 0.0 && p.nullvec_tol < 1.0) || !(p.coarse_tol_first > 0.0) || !(p.coarse_tol_rest > 0.0))
        return set_error("tolerances must be in (0, 1)"), MG_EINVAL;
    if (p.coarse_solver != MG_COARSE_DR_PROJ && p.coarse_solver != MG_COARSE_CGNE)
        return set_error("unknown coarse_solver %d", p.coarse_solver), MG_EINVAL;
    if (p.precision != MG_FP64 && p.precision != MG_MIXED && p.precision != MG_MIXED_BF16 &&
        p.precision != MG_MIXED_FP16)
        return set_error("unknown precision %d", p.precision), MG_EINVAL;
    if (p.rhs_block < 1 || p.rhs_block > 64) return set_error("rhs_block must be in [1, 64]"), MG_EINVAL;
    if ((p.precision == MG_MIXED_BF16 || p.precision == MG_MIXED_FP16) &&
        (p.method != MG_METHOD_MG || p.coarse_solver != MG_COARSE_DR_PROJ || p.partial_tol > 0.0))
        return set_error("the tensor-core block solve (precision %d) is built for the V-cycle with the deflated "
                         "coarse solve", p.precision), MG_EINVAL;
    if (p.method != MG_METHOD_MG && p.method != MG_METHOD_FINE_DEFLATION && p.method != MG_METHOD_FINE_CGNE)
        return set_error("unknown method %d", p.method), MG_EINVAL;
    if (p.method == MG_METHOD_FINE_CGNE && p.precision != MG_FP64)
        return set_error("the fine CGNE method runs in FP64 (precision MG_FP64)"), MG_EINVAL;
    if (p.dr_m - p.dr_k > MSMAX)
        return set_error("dr_m - dr_k must be <= %d", MSMAX), MG_EINVAL;
    if (!(p.partial_tol >= 0.0 && p.partial_tol < 1.0))
        return set_error("partial_tol must be in [0, 1)"), MG_EINVAL;
    if (p.partial_tol > 0.0 && (!(p.coarse_tol_partial > 0.0 && p.coarse_tol_partial < 1.0) || p.partial_max_iters < 1))
        return set_error("partial mode: coarse_tol_partial must be in (0, 1), partial_max_iters positive"),
               MG_EINVAL;
    if (p.pair_rhs != 0 && p.pair_rhs != 1) return set_error("pair_rhs must be 0 or 1"), MG_EINVAL;
    if (p.vcycle_graph != 0 && p.vcycle_graph != 1) return set_error("vcycle_graph must be 0 or 1"), MG_EINVAL;
    if (p.coarse_half != 0 && p.coarse_half != 1) return set_error("coarse_half must be 0 or 1"), MG_EINVAL;
    if (p.coarse_dcgs2 != 0 && p.coarse_dcgs2 != 1) return set_error("coarse_dcgs2 must be 0 or 1"), MG_EINVAL;
    if (p.lowrank_hops != 0 && p.lowrank_hops != 1) return set_error("lowrank_hops must be 0 or 1"), MG_EINVAL;
    if (p.coarse_mma != 0 && p.coarse_mma != 1) return set_error("coarse_mma must be 0 or 1"), MG_EINVAL;
    if (p.autotune != 0 && p.autotune != 1) return set_error("autotune must be 0 or 1"), MG_EINVAL;
    return MG_OK;
}

template <typename T>
mg_status alloc_level(Handle& H, Level<T>& L, int steps) {
    MG_TRY(halloc_t(H, &L.sV, (size_t)(steps + 1) * L.n));
    MG_TRY(halloc_t(H, &L.x, (size_t)L.n));
    MG_TRY(halloc_t(H, &L.f, (size_t)L.n));
    MG_TRY(halloc_t(H, &L.r, (size_t)L.n));
    MG_TRY(halloc_t(H, &L.ks, 1));
    return MG_OK;
}

template <typename T>
mg_status alloc_coarse(Handle& H, CoarseWS<T>& W, long n, int m, int k, bool own_defl) {
    MG_TRY(halloc_t(H, &W.V, (size_t)(m + 1) * n));
    MG_TRY(halloc_t(H, &W.V2, (size_t)(m + 1) * n));
    MG_TRY(halloc_t(H, &W.r, (size_t)n));
    MG_TRY(halloc_t(H, &W.p, (size_t)n));
    MG_TRY(halloc_t(H, &W.q, (size_t)n));
    MG_TRY(halloc_t(H, &W.t, (size_t)n));
    if (own_defl) MG_TRY(halloc_t(H, &W.W, (size_t)(k + 1) * n));
    MG_TRY(halloc_t(H, &W.ks, 1));
    return MG_OK;
}

// Every buffer a solve writes.  The owner of a hierarchy also holds the
// deflation spaces; a context made by make_context shares them.
mg_status alloc_workspaces(Handle& H, cudaStream_t s, bool owner) {
    const mg_params& p = H.p;
    const long n0 = H.L64[0].n, n2 = H.L64[2].n;
    H.red.max_blocks = 2 * sm_count();
    MG_TRY(halloc_t(H, &H.red.partial, (size_t)H.red.max_blocks * RED_MAXD));
    MG_TRY(halloc_t(H, &H.red.ticket, 1));
    MG_TRY(halloc_t(H, &H.sc, 1));
    MG_CUDA_TRY(cudaMemsetAsync(H.red.ticket, 0, sizeof(unsigned), s));
    MG_CUDA_TRY(cudaMemsetAsync(H.sc, 0, sizeof(Scalars), s));
    for (int l = 0; l < 3; ++l) {
        MG_TRY(alloc_level(H, H.L64[l], p.smooth_steps));
        MG_TRY(alloc_level(H, H.L32[l], p.smooth_steps));
    }
    MG_TRY(alloc_coarse(H, H.c64, n2, p.dr_m, p.dr_m, owner));
    MG_TRY(alloc_coarse(H, H.c32, n2, p.dr_m, p.dr_m, owner));
    MG_TRY(halloc_t(H, &H.fV, (size_t)(p.fgmres_m + 1) * n0));
    MG_TRY(halloc_t(H, &H.fZ, (size_t)p.fgmres_m * n0));
    MG_TRY(halloc_t(H, &H.fx, (size_t)n0));
    MG_TRY(halloc_t(H, &H.fr, (size_t)n0));
    MG_TRY(halloc_t(H, &H.fb, (size_t)n0));
    MG_TRY(halloc_t(H, &H.v32, (size_t)n0));
    MG_TRY(halloc_t(H, &H.z32, (size_t)n0));
    MG_TRY(halloc_t(H, &H.fks, 1));
    MG_TRY(halloc_t(H, &H.cvec, KLD));
    MG_TRY(halloc_t(H, &H.dvec, KLD));
    MG_TRY(halloc_t(H, &H.uvec, KLD));
    MG_TRY(halloc_t(H, &H.dr, 1));
    if (owner) MG_TRY(halloc_t(H, &H.pls, 1));
    H.cpart_ctas = sm_count();
    MG_TRY(halloc_t(H, &H.cpart, (size_t)2 * H.cpart_ctas * PSTR));
    MG_TRY(halloc_t(H, &H.cstats, 1));
    if (p.partial_tol > 0.0) {
        const long n1 = H.L64[1].n;
        MG_TRY(halloc_t(H, &H.p64.V, (size_t)(p.fgmres_m + 1) * n1));
        MG_TRY(halloc_t(H, &H.p64.Z, (size_t)p.fgmres_m * n1));
        MG_TRY(halloc_t(H, &H.p64.r, (size_t)n1));
        MG_TRY(halloc_t(H, &H.p64.ks, 1));
        MG_TRY(halloc_t(H, &H.p32.V, (size_t)(p.fgmres_m + 1) * n1));
        MG_TRY(halloc_t(H, &H.p32.Z, (size_t)p.fgmres_m * n1));
        MG_TRY(halloc_t(H, &H.p32.r, (size_t)n1));
        MG_TRY(halloc_t(H, &H.p32.ks, 1));
    }
    if (p.method == MG_METHOD_FINE_CGNE)
        for (int i = 0; i < 5; ++i) MG_TRY(halloc_t(H, &H.fcg[i], (size_t)n0));
    if (p.method == MG_METHOD_FINE_DEFLATION) {
        MG_TRY(halloc_t(H, &H.fdV, (size_t)(p.dr_m + 1) * n0));
        MG_TRY(halloc_t(H, &H.fdV2, (size_t)(p.dr_m + 1) * n0));
        MG_TRY(halloc_t(H, &H.fdks, 1));
        if (owner) {
            MG_TRY(halloc_t(H, &H.fdW, (size_t)(p.dr_m + 1) * n0));
            MG_TRY(halloc_t(H, &H.fdpls, 1));
        }
    }
    return MG_OK;
}

// Right-hand sides in lockstep pairs on two contexts A, B (pair_rhs): pairs
// p = p0, p0 + step, ... < npairs of the list first, first + 1, ... < nrhs, on
// stream s (device buffers).  Counters accumulate in A.st and B.st.  (Both
// right-hand sides of a pair run on one stream: splitting their V-cycles over
// two streams joined at the paired coarse kernel measured slower.)
mg_status solve_rhs_pairs(Handle& A, Handle& Bh, const double2* B, double2* X, int first, int nrhs, int p0, int step,
                          double tol, cudaStream_t s, int* iters, double* relres) {
    const long n0 = A.L64[0].n;
    MG_CUDA_TRY(cudaMemsetAsync(A.cstats, 0, sizeof(CoopStats), s));
    MG_CUDA_TRY(cudaMemsetAsync(Bh.cstats, 0, sizeof(CoopStats), s));
    mg_status result = MG_OK;
    const int npairs = (nrhs - first + 1) / 2;
    for (int p = p0; p < npairs; p += step) {
        const int i0 = first + 2 * p, i1 = i0 + 1;
        if (i1 >= nrhs) {  // an odd last one alone
            int it = 0;
            double rr = 0.0;
            bool conv = false;
            MG_TRY(fgmres_solve(A, B + (long)i0 * n0, X + (long)i0 * n0, tol, s, &it, &rr, &conv));
            if (iters) iters[i0] = it;
            if (relres) relres[i0] = rr;
            if (!conv) result = MG_ENOTCONV;
            continue;
        }
        Handle* HH[2] = {&A, &Bh};
        const double2* const bb[2] = {B + (long)i0 * n0, B + (long)i1 * n0};
        double2* const xx[2] = {X + (long)i0 * n0, X + (long)i1 * n0};
        int it[2] = {0, 0};
        double rr[2] = {0.0, 0.0};
        bool conv[2] = {false, false};
        MG_TRY(fgmres_solve_pair(HH, bb, xx, tol, s, it, rr, conv));
        for (int q = 0; q < 2; ++q) {
            const int i = q ? i1 : i0;
            if (iters) iters[i] = it[q];
            if (relres) relres[i] = rr[q];
            if (!conv[q]) result = MG_ENOTCONV;
        }
    }
    for (Handle* Hp : {&A, &Bh}) {
        CoopStats cs{};
        MG_CUDA_TRY(cudaMemcpyAsync(Hp->pinned, Hp->cstats, sizeof(CoopStats), cudaMemcpyDeviceToHost, s));
        MG_CUDA_TRY(cudaStreamSynchronize(s));
        std::memcpy(&cs, Hp->pinned, sizeof cs);
        Hp->st.coarse_iters += cs.iters;
        Hp->st.mvps[2] += cs.iters;
        if (cs.timeouts) return set_error("coarse solve: a bounded wait of the dataflow exchange gave up"), MG_ETIMEOUT;
    }
    return result;
}

// Solve right-hand sides i = i0, i0 + step, ... < i1 on handle (or context) H and
// stream s; counters accumulate in H.st.  Returns MG_ENOTCONV when one of them
// reached the iteration limit.
mg_status solve_rhs(Handle& H, const double2* B, double2* X, bool bdev, bool xdev, int i0, int i1, int step,
                    double tol, cudaStream_t s, int* iters, double* relres) {
    const long n0 = H.L64[0].n;
    if (H.is_context) {
        const bool needs = H.p.method == MG_METHOD_FINE_DEFLATION || H.p.coarse_solver == MG_COARSE_DR_PROJ;
        const int k = H.p.method == MG_METHOD_FINE_DEFLATION ? H.fine_k : H.defl_k;
        if (needs && k == 0) return set_error("a solve context cannot build the deflation space"), MG_EINVAL;
    }
    MG_CUDA_TRY(cudaMemsetAsync(H.cstats, 0, sizeof(CoopStats), s));
    mg_status result = MG_OK;
    for (int i = i0; i < i1; i += step) {
        const double2* bi = B + (long)i * n0;
        double2* xi = X + (long)i * n0;
        const double2* bsrc = bi;
        double2* xdst = xi;
        if (!bdev) {
            MG_CUDA_TRY(cudaMemcpyAsync(H.fb, bi, n0 * sizeof(double2), cudaMemcpyHostToDevice, s));
            bsrc = H.fb;
        }
        if (!xdev) xdst = H.fx;
        int it = 0;
        double rr = 0.0;
        bool conv = false;
        if (H.p.method == MG_METHOD_FINE_DEFLATION)
            MG_TRY(fine_deflated_solve(H, bsrc, xdst, tol, s, &it, &rr, &conv));
        else if (H.p.method == MG_METHOD_FINE_CGNE)
            MG_TRY(fine_cgne_solve(H, bsrc, xdst, tol, s, &it, &rr, &conv));
        else
            MG_TRY(fgmres_solve(H, bsrc, xdst, tol, s, &it, &rr, &conv));
        if (!xdev) MG_CUDA_TRY(cudaMemcpyAsync(xi, H.fx, n0 * sizeof(double2), cudaMemcpyDeviceToHost, s));
        if (iters) iters[i] = it;
        if (relres) relres[i] = rr;
        if (!conv) result = MG_ENOTCONV;
    }
    CoopStats cs{};
    MG_CUDA_TRY(cudaMemcpyAsync(H.pinned, H.cstats, sizeof(CoopStats), cudaMemcpyDeviceToHost, s));
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(&cs, H.pinned, sizeof cs);
    H.st.coarse_iters += cs.iters;
    H.st.mvps[2] += cs.iters;
    if (cs.timeouts) return set_error("coarse solve: a bounded wait of the dataflow exchange gave up"), MG_ETIMEOUT;
    return result;
}

// A solve context of hierarchy P: the same (read-only) hierarchy and deflation
// spaces, its own workspaces and stream, so that right-hand sides can be solved
// concurrently.  Requires the deflation space of P to exist.
mg_status make_context(Handle& P, mg_handle_s** out) {
    *out = nullptr;
    mg_handle_s* cs = new (std::nothrow) mg_handle_s();
    if (!cs) return set_error("out of host memory"), MG_ENOMEM;
    Handle& C = cs->h;
    C.Lx = P.Lx;
    C.Lt = P.Lt;
    C.m0 = P.m0;
    C.p = P.p;
    C.is_context = true;
    for (int l = 0; l < 3; ++l) {
        C.L64[l] = P.L64[l];
        C.L32[l] = P.L32[l];
        C.L64[l].timer = C.L32[l].timer = &C.timers[l];
    }
    C.U64 = P.U64;
    C.U32 = P.U32;
    for (int l = 0; l < 3; ++l) {
        C.A64[l] = P.A64[l];
        C.A32[l] = P.A32[l];
    }
    C.A16c = P.A16c;
    for (int l = 0; l < 2; ++l) {
        C.Q64[l] = P.Q64[l];
        C.Q32[l] = P.Q32[l];
    }
    C.c64.W = P.c64.W;
    C.c32.W = P.c32.W;
    C.pls = P.pls;
    C.defl_k = P.defl_k;
    C.fdW = P.fdW;
    C.fdpls = P.fdpls;
    C.fine_k = P.fine_k;
    auto fail = [&](mg_status st) {
        for (void* q : C.allocs) cudaFree(q);
        if (C.pinned) cudaFreeHost(C.pinned);
        if (C.own_stream) cudaStreamDestroy(C.own_stream);
        delete cs;
        return st;
    };
    if (cudaMallocHost(&C.pinned, 1 << 16) != cudaSuccess) {
        (void)cudaGetLastError();
        C.pinned = nullptr;
        set_error("cudaMallocHost failed");
        return fail(MG_ENOMEM);
    }
    if (cudaStreamCreateWithFlags(&C.own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        C.own_stream = nullptr;
        set_error("cudaStreamCreate failed");
        return fail(MG_ECUDA);
    }
    mg_status st = alloc_workspaces(C, C.own_stream, false);
    if (st != MG_OK) return fail(st);
    if (cudaStreamSynchronize(C.own_stream) != cudaSuccess) {
        set_error("context set-up failed");
        return fail(MG_ECUDA);
    }
    *out = cs;
    return MG_OK;
}

// Gaussian start vectors (E|z|^2 = 1) from a counter hash of (seed, grid, index)
void host_gaussian(std::vector<double>& out, size_t ncomplex, unsigned long long seed, int grid) {
    out.resize(2 * ncomplex);
    auto mix = [](unsigned long long z) {
        z += 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    const unsigned long long key = mix(seed ^ (0xA5A5ULL + (unsigned long long)grid * 0x1000193ULL));
    for (size_t i = 0; i < ncomplex; ++i) {
        const double u1 = ((double)(mix(key ^ mix(2 * i)) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((double)(mix(key ^ mix(2 * i + 1)) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double rad = std::sqrt(-std::log(u1));  // |z|^2 ~ Exp(1)
        out[2 * i] = rad * std::cos(6.283185307179586 * u2);
        out[2 * i + 1] = rad * std::sin(6.283185307179586 * u2);
    }
}

mg_status setup_common(const void* gauge, int Lx, int Lt, double m0, int nvec, int block, const mg_params* pp,
                       const void* starts0, const void* starts1, const void* nv0, const void* nv1, void* stream,
                       mg_handle* out) {
    if (!out) return set_error("out is NULL"), MG_EINVAL;
    *out = nullptr;
    if (!gauge) return set_error("gauge is NULL"), MG_EINVAL;
    mg_params p;
    mg_default_params(&p);
    if (pp) p = *pp;
    if (nvec != p.nvec || block != p.block)
        return set_error("nvec/block (%d, %d) differ from the parameters (%d, %d)", nvec, block, p.nvec, p.block),
               MG_EINVAL;
    MG_TRY(check_params(p));
    if (Lx < 16 || Lt < 16 || Lx % 16 || Lt % 16)
        return set_error("lattice %d x %d: both extents must be positive multiples of 16", Lx, Lt), MG_EINVAL;
    if ((long)Lx * Lt > (1L << 26)) return set_error("lattice too large"), MG_EINVAL;
    if (!std::isfinite(m0)) return set_error("m0 is not finite"), MG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mg_handle_s* hs = new (std::nothrow) mg_handle_s();
    if (!hs) return set_error("out of host memory"), MG_ENOMEM;
    Handle& H = hs->h;
    H.Lx = Lx;
    H.Lt = Lt;
    H.m0 = m0;
    H.p = p;
    auto fail = [&](mg_status st) {
        free_handle(H);
        delete hs;
        return st;
    };
    if (cudaMallocHost(&H.pinned, 1 << 16) != cudaSuccess) {
        (void)cudaGetLastError();
        H.pinned = nullptr;
        set_error("cudaMallocHost failed");
        return fail(MG_ENOMEM);
    }
    // grids
    const int nx[3] = {Lx, Lx / 4, Lx / 16}, nt[3] = {Lt, Lt / 4, Lt / 16}, dof[3] = {2, 24, 24};
    for (int l = 0; l < 3; ++l) {
        H.L64[l].Nx = H.L32[l].Nx = nx[l];
        H.L64[l].Nt = H.L32[l].Nt = nt[l];
        H.L64[l].dof = H.L32[l].dof = dof[l];
        H.L64[l].n = H.L32[l].n = (long)nx[l] * nt[l] * dof[l];
        H.L64[l].h = H.L32[l].h = dof[l] / 2;
        H.L64[l].m0 = H.L32[l].m0 = m0;
        H.L64[l].timer = H.L32[l].timer = &H.timers[l];
    }
    const long n0 = H.L64[0].n;
    mg_status st;
#define TRYF(e)                     \
    do {                            \
        st = (e);                   \
        if (st != MG_OK) return fail(st); \
    } while (0)
    // hierarchy buffers
    TRYF(halloc_t(H, &H.U64, (size_t)2 * Lx * Lt));
    TRYF(halloc_t(H, &H.U32, (size_t)2 * Lx * Lt));
    for (int l = 1; l < 3; ++l) {
        TRYF(halloc_t(H, &H.A64[l], (size_t)nx[l] * nt[l] * 5 * 576));
        TRYF(halloc_t(H, &H.A32[l], (size_t)nx[l] * nt[l] * 5 * 576));
    }
    if (p.precision != MG_FP64 && p.coarse_half) TRYF(halloc_t(H, &H.A16c, (size_t)nx[2] * nt[2] * 5 * 576));
    if (p.lowrank_hops) {
        TRYF(halloc_t(H, &H.F64, (size_t)nx[1] * nt[1] * LR_SITE));
        TRYF(halloc_t(H, &H.F32, (size_t)nx[1] * nt[1] * LR_SITE));
    }
    for (int l = 0; l < 2; ++l) {
        const size_t q = (size_t)nx[l + 1] * nt[l + 1] * 24 * 16 * (dof[l] / 2);
        TRYF(halloc_t(H, &H.Q64[l], q));
        TRYF(halloc_t(H, &H.Q32[l], q));
    }
    H.L64[0].U = H.U64;
    H.L32[0].U = H.U32;
    for (int l = 1; l < 3; ++l) {
        H.L64[l].A = H.A64[l];
        H.L32[l].A = H.A32[l];
    }
    for (int l = 0; l < 2; ++l) {
        H.L64[l].Q = H.Q64[l];
        H.L32[l].Q = H.Q32[l];
    }
    TRYF(alloc_workspaces(H, s, true));
    if (cudaMemcpyAsync(H.U64, gauge, sizeof(double2) * 2 * Lx * Lt, cudaMemcpyDefault, s) != cudaSuccess) {
        set_error("copy of the gauge field failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(MG_ECUDA);
    }
    // start vectors of the near-null solves
    std::vector<double> g0, g1;
    const long n1 = H.L64[1].n;
    double2* d_starts[2] = {nullptr, nullptr};
    if (!nv0 || !nv1) {
        const void* src[2] = {starts0, starts1};
        const long nn[2] = {n0, n1};
        for (int l = 0; l < 2; ++l) {
            TRYF(halloc_t(H, &d_starts[l], (size_t)p.nvec * nn[l]));
            if (src[l]) {
                if (cudaMemcpyAsync(d_starts[l], src[l], sizeof(double2) * p.nvec * nn[l], cudaMemcpyDefault, s) !=
                    cudaSuccess) {
                    set_error("copy of start vectors failed");
                    return fail(MG_ECUDA);
                }
            } else {
                std::vector<double>& g = (l == 0) ? g0 : g1;
                host_gaussian(g, (size_t)p.nvec * nn[l], p.seed, l);
                if (cudaMemcpyAsync(d_starts[l], g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess) {
                    set_error("copy of start vectors failed");
                    return fail(MG_ECUDA);
                }
            }
        }
    }
    const double2* nvd[2] = {nullptr, nullptr};
    if (nv0 && nv1) {
        nvd[0] = static_cast<const double2*>(nv0);
        nvd[1] = static_cast<const double2*>(nv1);
    }
    TRYF(build_hierarchy(H, H.U64, d_starts[0], d_starts[1], nvd[0], nvd[1], s));
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(MG_ECUDA);
    }
    if (p.autotune) TRYF(tune_shapes(H, s));
#undef TRYF
    *out = hs;
    return MG_OK;
}

}  // namespace

mg_status make_solve_context(mg_handle_s* owner, mg_handle_s** out) {
    if (!owner || owner->h.is_context) return set_error("a solve context needs a hierarchy owner"), MG_EINVAL;
    return make_context(owner->h, out);
}
size_t handle_device_bytes(const mg_handle_s* h) { return h ? h->h.bytes : 0; }
cudaStream_t handle_stream(const mg_handle_s* h) { return h ? h->h.own_stream : nullptr; }

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_default_params(mg_params* p) {
    if (!p) return set_error("p is NULL"), MG_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->levels = 3;
    p->block = 4;
    p->nvec = 12;
    p->smooth_steps = 2;
    p->fgmres_m = 8;
    p->max_outer = 500;
    p->coarse_solver = MG_COARSE_DR_PROJ;
    p->dr_m = 30;
    p->dr_k = 10;
    p->dr_max_cycles = 100;
    p->dr_stall_cycles = 2;
    p->proj_max_cycles = 1000;
    p->cgne_max_iters = 100000;
    p->nullvec_max_iters = 100000;
    p->nullvec_tol = 1e-4;
    p->coarse_tol_first = 1e-14;
    p->coarse_tol_rest = 1e-8;
    p->precision = MG_FP64;
    p->seed = 12345ULL;
    p->method = MG_METHOD_MG;
    p->parallel = 1;
    p->partial_tol = 0.0;
    p->coarse_tol_partial = 1e-2;
    p->partial_max_iters = 200;
    p->pair_rhs = 0;
    p->vcycle_graph = 1;
    p->coarse_half = 1;
    p->coarse_dcgs2 = 0;
    p->rhs_block = 64;
    p->lowrank_hops = 1;
    p->coarse_mma = 1;
    p->autotune = 1;
    return MG_OK;
}

const char* mg_last_error(void) { return g_last_error.c_str(); }

mg_status mg_setup(const void* gauge, int L_x, int L_t, double m0, int nvec, int block, const mg_params* p,
                   const void* starts0, const void* starts1, void* stream, mg_handle* out) {
    try {
        return setup_common(gauge, L_x, L_t, m0, nvec, block, p, starts0, starts1, nullptr, nullptr, stream, out);
    } catch (const std::bad_alloc&) {
        set_error("out of host memory");
        return MG_ENOMEM;
    }
}

mg_status mg_setup_from_vectors(const void* gauge, int L_x, int L_t, double m0, int nvec, int block,
                                const mg_params* p, const void* nullvecs0, const void* nullvecs1, void* stream,
                                mg_handle* out) {
    if (!nullvecs0 || !nullvecs1) return set_error("nullvecs0/1 must not be NULL"), MG_EINVAL;
    try {
        return setup_common(gauge, L_x, L_t, m0, nvec, block, p, nullptr, nullptr, nullvecs0, nullvecs1, stream,
                            out);
    } catch (const std::bad_alloc&) {
        set_error("out of host memory");
        return MG_ENOMEM;
    }
}

mg_status mg_destroy(mg_handle h) {
    if (!h) return MG_OK;
    free_handle(h->h);
    delete h;
    return MG_OK;
}

mg_status mg_reset_deflation(mg_handle h) {
    if (!h) return set_error("handle is NULL"), MG_EINVAL;
    h->h.defl_k = 0;
    h->h.fine_k = 0;
    return MG_OK;
}

mg_status mg_solve(mg_handle h, const void* b, void* x, int nrhs, double tol, void* stream, int* iters,
                   double* relres, mg_solve_stats* stats) {
    if (!h) return set_error("handle is NULL"), MG_EINVAL;
    if (!b || !x) return set_error("b or x is NULL"), MG_EINVAL;
    if (nrhs < 0) return set_error("nrhs < 0"), MG_EINVAL;
    if (!(tol > 0.0) || !(tol < 1.0)) return set_error("tol must be in (0, 1)"), MG_EINVAL;
    if (b == x) return set_error("b and x must not alias"), MG_EINVAL;
    Handle& H = h->h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    H.st = Stats{};
    const long n0 = H.L64[0].n;
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    const double2* B = static_cast<const double2*>(b);
    double2* X = static_cast<double2*>(x);
    const bool have_defl = (H.p.method == MG_METHOD_FINE_DEFLATION) ? H.fine_k > 0 : H.defl_k > 0;
    const bool needs_defl = H.p.method == MG_METHOD_FINE_DEFLATION || H.p.coarse_solver == MG_COARSE_DR_PROJ;
    int par = std::min(nrhs, std::max(H.p.parallel, 1));
    bool notconv = false;
    auto seq = [&](int i0, int i1) -> mg_status {
        const mg_status r = solve_rhs(H, B, X, bdev, xdev, i0, i1, 1, tol, s, iters, relres);
        if (r == MG_ENOTCONV) notconv = true;
        return r == MG_ENOTCONV ? MG_OK : r;
    };
    // precision MG_MIXED_BF16 / MG_MIXED_FP16: lockstep blocks of rhs_block right-hand
    // sides with tensor-core block products, after the first right-hand side of the
    // handle has built the deflation space alone (FP32 path, FP64 GMRES-DR)
    const bool block = (H.p.precision == MG_MIXED_BF16 || H.p.precision == MG_MIXED_FP16) && !H.is_context;
    if (block) {
        int first = 0;
        if (!have_defl) {
            MG_TRY(seq(0, std::min(nrhs, 1)));
            first = 1;
        }
        for (int i0 = first; i0 < nrhs; i0 += H.p.rhs_block) {
            const int nb = std::min(H.p.rhs_block, nrhs - i0);
            std::vector<int> it(nb, 0);
            std::vector<double> rr(nb, 0.0);
            std::unique_ptr<bool[]> cv(new bool[nb]);
            MG_TRY(fgmres_solve_block(H, B + (long)i0 * n0, X + (long)i0 * n0, nb, tol,
                                      H.p.precision == MG_MIXED_FP16, s, it.data(), rr.data(), cv.get(), nullptr));
            for (int r = 0; r < nb; ++r) {
                if (iters) iters[i0 + r] = it[r];
                if (relres) relres[i0 + r] = rr[r];
                if (!cv[r]) notconv = true;
            }
        }
    } else if (par <= 1) {
        MG_TRY(seq(0, nrhs));
    } else {
        // the first right-hand side builds the deflation space alone; the rest are
        // spread over `par` concurrent contexts (this handle + par - 1 contexts)
        int first = 0;
        if (needs_defl && !have_defl) {
            MG_TRY(seq(0, 1));
            first = 1;
            par = std::min(par, nrhs - 1);
        }
        if (first < nrhs) {
            // pair_rhs: every worker drives two contexts in lockstep
            const bool pairs = H.p.pair_rhs && H.p.precision == MG_MIXED && H.p.method == MG_METHOD_MG &&
                               H.p.coarse_solver == MG_COARSE_DR_PROJ && H.p.partial_tol == 0.0 && bdev && xdev;
            if (pairs) par = std::max(1, std::min(par, (nrhs - first + 1) / 2));
            const int nctx = pairs ? 2 * par - 1 : par - 1;
            while ((int)H.contexts.size() < nctx) {
                mg_handle_s* c = nullptr;
                MG_TRY(make_context(H, &c));
                H.contexts.push_back(c);
            }
            for (mg_handle_s* c : H.contexts) {  // a context created before a deflation reset
                c->h.defl_k = H.defl_k;
                c->h.fine_k = H.fine_k;
            }
            // this handle's share runs on a non-blocking stream of its own, like the
            // contexts' (not on the caller's stream, which may be the legacy default
            // stream); inputs written on the caller's stream must be visible to all
            if (!H.work_stream) MG_CUDA_TRY(cudaStreamCreateWithFlags(&H.work_stream, cudaStreamNonBlocking));
            const cudaStream_t ws = H.work_stream;
            cudaEvent_t ev;
            MG_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            MG_CUDA_TRY(cudaEventRecord(ev, s));
            MG_CUDA_TRY(cudaStreamWaitEvent(ws, ev, 0));
            for (int w = 0; w < nctx; ++w) MG_CUDA_TRY(cudaStreamWaitEvent(H.contexts[w]->h.own_stream, ev, 0));
            std::vector<mg_status> st_w(par, MG_OK);
            std::vector<std::string> err_w(par);
            std::vector<std::thread> th;
            int dev = 0;
            MG_CUDA_TRY(cudaGetDevice(&dev));
            for (int w = 1; w < par; ++w) {
                th.emplace_back([&, w]() {
                    cudaSetDevice(dev);
                    if (pairs) {
                        Handle& C = H.contexts[2 * w - 1]->h;
                        Handle& D = H.contexts[2 * w]->h;
                        C.st = Stats{};
                        D.st = Stats{};
                        st_w[w] = solve_rhs_pairs(C, D, B, X, first, nrhs, w, par, tol, C.own_stream, iters, relres);
                    } else {
                        Handle& C = H.contexts[w - 1]->h;
                        C.st = Stats{};
                        st_w[w] =
                            solve_rhs(C, B, X, bdev, xdev, first + w, nrhs, par, tol, C.own_stream, iters, relres);
                    }
                    if (st_w[w] != MG_OK && st_w[w] != MG_ENOTCONV) err_w[w] = mg_last_error();
                });
            }
            const Stats keep = H.st;  // the first right-hand side, if it ran alone
            H.st = Stats{};
            if (pairs) {
                Handle& D = H.contexts[0]->h;
                D.st = Stats{};
                st_w[0] = solve_rhs_pairs(H, D, B, X, first, nrhs, 0, par, tol, ws, iters, relres);
            } else {
                st_w[0] = solve_rhs(H, B, X, bdev, xdev, first, nrhs, par, tol, ws, iters, relres);
            }
            for (auto& t : th) t.join();
            // later work on the caller's stream follows every worker's
            cudaEventRecord(ev, ws);
            cudaStreamWaitEvent(s, ev, 0);
            for (int w = 0; w < nctx; ++w) {
                cudaEventRecord(ev, H.contexts[w]->h.own_stream);
                cudaStreamWaitEvent(s, ev, 0);
            }
            cudaEventDestroy(ev);
            Stats sum = keep;
            for (int w = 0; w <= nctx; ++w) {
                const Stats& sw = (w == 0) ? H.st : H.contexts[w - 1]->h.st;
                for (int l = 0; l < 3; ++l) sum.mvps[l] += sw.mvps[l];
                sum.outer += sw.outer;
                sum.coarse_solves += sw.coarse_solves;
                sum.coarse_iters += sw.coarse_iters;
                sum.dr_solves += sw.dr_solves;
            }
            H.st = sum;
            for (int w = 0; w < par; ++w) {
                if (st_w[w] != MG_OK && st_w[w] != MG_ENOTCONV) {
                    if (!err_w[w].empty()) set_error("%s", err_w[w].c_str());
                    return st_w[w];
                }
            }
            for (int w = 0; w < par; ++w)
                if (st_w[w] == MG_ENOTCONV) notconv = true;
        }
    }
    MG_CUDA_TRY(cudaGetLastError());
    const mg_status result = notconv ? MG_ENOTCONV : MG_OK;
    if (stats) {
        for (int l = 0; l < 3; ++l) stats->mvps[l] = H.st.mvps[l];
        const double n1 = (double)H.L64[1].n, n2 = (double)H.L64[2].n, nf = (double)n0;
        stats->fine_equiv_mvps = H.st.mvps[0] + n1 / nf * H.st.mvps[1] + n2 / nf * H.st.mvps[2];
        stats->outer_iters = H.st.outer;
        stats->coarse_solves = H.st.coarse_solves;
        stats->coarse_iters = H.st.coarse_iters;
        stats->dr_solves = H.st.dr_solves;
    }
    if (result == MG_ENOTCONV) set_error("some right-hand side reached max_outer");
    return result;
}

mg_status mg_level_shape(mg_handle h, int level, int* n_x, int* n_t, int* dof) {
    if (!h || level < 0 || level > 2) return set_error("bad handle or level"), MG_EINVAL;
    const Level<double>& L = h->h.L64[level];
    if (n_x) *n_x = L.Nx;
    if (n_t) *n_t = L.Nt;
    if (dof) *dof = L.dof;
    return MG_OK;
}

mg_status mg_stencil_info(mg_handle h, int level, int* factored, double* max_rel_err) {
    if (!h || level < 1 || level > 2 || !factored) return set_error("bad handle, level or output"), MG_EINVAL;
    const Handle& H = h->h;
    *factored = H.L64[level].F ? 1 : 0;
    if (max_rel_err) *max_rel_err = H.L64[level].F ? H.lowrank_err : 0.0;
    return MG_OK;
}

mg_status mg_launch_shape(mg_handle h, int level, int precision, int* shape, double* us) {
    if (!h || level < 0 || level > 2 || !shape) return set_error("bad handle, level or output"), MG_EINVAL;
    if (precision != MG_F64 && precision != MG_F32) return set_error("precision must be MG_F64 or MG_F32"), MG_EINVAL;
    const Handle& H = h->h;
    const int sh = precision == MG_F64 ? H.L64[level].shape : H.L32[level].shape;
    const double* t = precision == MG_F64 ? H.L64[level].shape_us : H.L32[level].shape_us;
    *shape = sh;
    if (us) {
        us[0] = t[0];
        us[1] = t[1];
    }
    return MG_OK;
}

mg_status mg_set_launch_shape(mg_handle h, int level, int precision, int shape) {
    if (!h || level < 0 || level > 2) return set_error("bad handle or level"), MG_EINVAL;
    if (precision != MG_F64 && precision != MG_F32) return set_error("precision must be MG_F64 or MG_F32"), MG_EINVAL;
    Handle& H = h->h;
    if (H.is_context) return set_error("a solve context takes its owner's shapes"), MG_EINVAL;
    const bool f32 = precision == MG_F32;
    const bool wil = level == 0, lr = f32 ? H.L32[level].F != nullptr : false;
    const int* cand = wil ? WILSON_SHAPES : lr ? STENCIL_LR_F32_SHAPES : STENCIL_F32_SHAPES;
    const int nc = wil ? (int)(sizeof(WILSON_SHAPES) / sizeof(int))
                       : lr ? (int)(sizeof(STENCIL_LR_F32_SHAPES) / sizeof(int))
                            : (int)(sizeof(STENCIL_F32_SHAPES) / sizeof(int));
    bool ok = shape == 0;
    if (wil || f32)
        for (int i = 0; i < nc; ++i) ok = ok || shape == cand[i];
    if (!ok) return set_error("shape %d is not a candidate of this apply", shape), MG_EINVAL;
    (f32 ? H.L32[level].shape : H.L64[level].shape) = shape;
    if (H.vg.exec) {  // a captured V-cycle keeps the shapes it was captured with: capture again
        cudaGraphExecDestroy(H.vg.exec);
        H.vg = VGraph{};
    }
    return MG_OK;
}

mg_status mg_apply(mg_handle h, int level, int dagger, int precision, const void* x, void* y, void* stream) {
    if (!h || level < 0 || level > 2) return set_error("bad handle or level"), MG_EINVAL;
    if (!x || !y || x == y) return set_error("x, y must be distinct device pointers"), MG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == MG_F64)
        h->h.L64[level].apply(static_cast<double2*>(y), static_cast<const double2*>(x), nullptr, dagger != 0, Gate{}, s);
    else if (precision == MG_F32)
        h->h.L32[level].apply(static_cast<float2*>(y), static_cast<const float2*>(x), nullptr, dagger != 0, Gate{}, s);
    else
        return set_error("unknown precision"), MG_EINVAL;
    MG_LAUNCH_CHECK();
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status mg_restrict(mg_handle h, int level, int precision, const void* fine, void* coarse, void* stream) {
    if (!h || level < 0 || level > 1) return set_error("bad handle or level"), MG_EINVAL;
    if (!fine || !coarse) return set_error("NULL vector"), MG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Handle& H = h->h;
    if (precision == MG_F64) {
        const Level<double>& L = H.L64[level];
        launch_restrict<double>(static_cast<double2*>(coarse), static_cast<const double2*>(fine), L.Q, L.Nx, L.Nt,
                                L.h, Gate{}, s);
    } else if (precision == MG_F32) {
        const Level<float>& L = H.L32[level];
        launch_restrict<float>(static_cast<float2*>(coarse), static_cast<const float2*>(fine), L.Q, L.Nx, L.Nt, L.h,
                               Gate{}, s);
    } else {
        return set_error("unknown precision"), MG_EINVAL;
    }
    MG_LAUNCH_CHECK();
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status mg_prolong(mg_handle h, int level, int precision, const void* coarse, void* fine, void* stream) {
    if (!h || level < 0 || level > 1) return set_error("bad handle or level"), MG_EINVAL;
    if (!fine || !coarse) return set_error("NULL vector"), MG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Handle& H = h->h;
    if (precision == MG_F64) {
        const Level<double>& L = H.L64[level];
        launch_prolong<double>(static_cast<double2*>(fine), static_cast<const double2*>(coarse), L.Q, L.Nx, L.Nt,
                               L.h, false, Gate{}, s);
    } else if (precision == MG_F32) {
        const Level<float>& L = H.L32[level];
        launch_prolong<float>(static_cast<float2*>(fine), static_cast<const float2*>(coarse), L.Q, L.Nx, L.Nt, L.h,
                              false, Gate{}, s);
    } else {
        return set_error("unknown precision"), MG_EINVAL;
    }
    MG_LAUNCH_CHECK();
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status mg_get_stencil(mg_handle h, int level, void* out) {
    if (!h || level < 1 || level > 2 || !out) return set_error("bad handle, level or pointer"), MG_EINVAL;
    const Handle& H = h->h;
    const Level<double>& L = H.L64[level];
    const size_t nblk = (size_t)L.Nx * L.Nt * 5;
    std::vector<double2> tmp(nblk * 576), tr(nblk * 576);
    MG_CUDA_TRY(cudaMemcpy(tmp.data(), H.A64[level], tmp.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    // device blocks are column-major [l][k]; the ABI returns row-major [k][l]
    for (size_t b = 0; b < nblk; ++b)
        for (int k = 0; k < 24; ++k)
            for (int l = 0; l < 24; ++l) tr[b * 576 + k * 24 + l] = tmp[b * 576 + l * 24 + k];
    MG_CUDA_TRY(cudaMemcpy(out, tr.data(), tr.size() * sizeof(double2), cudaMemcpyDefault));
    return MG_OK;
}

mg_status mg_get_prolongator(mg_handle h, int level, void* out) {
    if (!h || level < 0 || level > 1 || !out) return set_error("bad handle, level or pointer"), MG_EINVAL;
    const Handle& H = h->h;
    const size_t q = (size_t)H.L64[level + 1].Nx * H.L64[level + 1].Nt * 24 * 16 * H.L64[level].h;
    MG_CUDA_TRY(cudaMemcpy(out, H.Q64[level], q * sizeof(double2), cudaMemcpyDefault));
    return MG_OK;
}

mg_status mg_get_deflation(mg_handle h, void* W, void* Hm, int* k_out) {
    if (!h) return set_error("handle is NULL"), MG_EINVAL;
    const Handle& H = h->h;
    const int k = H.defl_k;
    if (k_out) *k_out = k;
    if (k == 0) return MG_OK;
    const long n2 = H.L64[2].n;
    if (W) MG_CUDA_TRY(cudaMemcpy(W, H.c64.W, (size_t)(k + 1) * n2 * sizeof(double2), cudaMemcpyDefault));
    if (Hm) {
        std::vector<double2> colmaj((size_t)KLD * KMAX), rowmaj((size_t)(k + 1) * k);
        MG_CUDA_TRY(cudaMemcpy(colmaj.data(), MG_DEVF(H.pls, double2, H), colmaj.size() * sizeof(double2),
                               cudaMemcpyDeviceToHost));
        for (int i = 0; i <= k; ++i)
            for (int j = 0; j < k; ++j) rowmaj[(size_t)i * k + j] = colmaj[(size_t)i + (size_t)KLD * j];
        MG_CUDA_TRY(cudaMemcpy(Hm, rowmaj.data(), rowmaj.size() * sizeof(double2), cudaMemcpyDefault));
    }
    return MG_OK;
}

mg_status mg_timing_enable(mg_handle h, int level, int enable) {
    if (!h || level < 0 || level > 2) return set_error("bad handle or level"), MG_EINVAL;
    ApplyTimer& t = h->h.timers[level];
    t.on = enable != 0;
    t.used = 0;
    return MG_OK;
}

mg_status mg_timing_read(mg_handle h, int level, double* total_ms, long long* launches) {
    if (!h || level < 0 || level > 2) return set_error("bad handle or level"), MG_EINVAL;
    ApplyTimer& t = h->h.timers[level];
    double ms = 0.0;
    if (t.used >= 2) MG_CUDA_TRY(cudaEventSynchronize(t.ev[t.used - 1]));
    for (size_t i = 0; i + 1 < t.used; i += 2) {
        float v = 0.f;
        MG_CUDA_TRY(cudaEventElapsedTime(&v, t.ev[i], t.ev[i + 1]));
        ms += v;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = (long long)(t.used / 2);
    return MG_OK;
}

unsigned long long mg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

mg_status mg_wilson_apply(const void* gauge, int L_x, int L_t, double m0, int dagger, int precision, const void* x,
                          void* y, void* stream) {
    if (!gauge || !x || !y || x == y) return set_error("gauge, x, y must be distinct non-NULL pointers"), MG_EINVAL;
    if (L_x < 2 || L_t < 2) return set_error("lattice extents must be >= 2"), MG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == MG_F64)
        launch_wilson<double>(static_cast<double2*>(y), static_cast<const double2*>(x),
                              static_cast<const double2*>(gauge), nullptr, m0, L_x, L_t, dagger != 0, Gate{}, s);
    else if (precision == MG_F32)
        launch_wilson<float>(static_cast<float2*>(y), static_cast<const float2*>(x), static_cast<const float2*>(gauge),
                             nullptr, m0, L_x, L_t, dagger != 0, Gate{}, s);
    else
        return set_error("unknown precision"), MG_EINVAL;
    MG_LAUNCH_CHECK();
    return MG_OK;
}

}  // extern "C"
