// C ABI of the coarsest grid alone: load a deflation space into a handle, and
// run one projected coarse solve (GMRES-Proj, Section 2) on the handle's
// coarsest operator with the launch shape the V-cycle uses.  Both exist so that
// the coarse solve can be compared with an independent implementation on
// identical inputs, at the geometry the solver runs at full size.
#include <cstring>
#include <vector>

#include "handle.cuh"

using namespace mg;

namespace {

mg_status device_vectors(const void* p, const char* what) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error("%s must be device memory", what), MG_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error("%s must be device memory", what), MG_EINVAL;
    return MG_OK;
}

template <typename T>
CoopArgs<T> coarse_args(Handle& H, const C2<T>* f, C2<T>* x, C2<T>* r, C2<T>* V, double2* part, int part_ctas,
                        CoopStats* out, double tol) {
    const Level<T>& L = H.levels<T>()[2];
    CoopArgs<T> a{};
    a.A = L.A;
    a.Nx = L.Nx;
    a.Nt = L.Nt;
    a.f = f;
    a.x = x;
    a.r = r;
    a.V = V;
    a.W = H.coarse<T>().W;
    a.pls = H.pls;
    a.k = H.defl_k;
    a.ms = std::max(H.p.dr_m - H.defl_k, 1);
    a.tol = tol;
    a.max_cycles = H.p.proj_max_cycles;
    a.part = part;
    a.part_ctas = part_ctas;
    a.out = out;
    a.Ah = std::is_same<T, float>::value ? H.A16c : nullptr;
    a.dc = H.p.coarse_dcgs2;
    a.mma = H.p.coarse_mma;
    return a;
}

}  // namespace

extern "C" {

mg_status mg_set_deflation(mg_handle h, const void* W, const void* Hm, int k) {
    if (!h || !W || !Hm) return set_error("handle, W and H must be non-NULL"), MG_EINVAL;
    Handle& H = h->h;
    if (H.is_context) return set_error("a solve context shares its owner's deflation space"), MG_EINVAL;
    if (k < 1 || k > H.p.dr_m || k + 1 > PSTR || k > KMAX - 1)
        return set_error("deflation size k = %d must be in [1, dr_m = %d]", k, H.p.dr_m), MG_EINVAL;
    const long n2 = H.L64[2].n;
    cudaStream_t s = nullptr;
    // W rows as given; H_k row-major (k+1) x k into the column-major layout of the factored state
    MG_CUDA_TRY(cudaMemcpy(H.c64.W, W, (size_t)(k + 1) * n2 * sizeof(double2), cudaMemcpyDefault));
    std::vector<double2> rowmaj((size_t)(k + 1) * k), colmaj((size_t)KLD * KMAX);
    MG_CUDA_TRY(cudaMemcpy(rowmaj.data(), Hm, rowmaj.size() * sizeof(double2), cudaMemcpyDefault));
    for (auto& z : colmaj) z = make_double2(0.0, 0.0);
    for (int i = 0; i <= k; ++i)
        for (int j = 0; j < k; ++j) colmaj[(size_t)i + (size_t)KLD * j] = rowmaj[(size_t)i * k + j];
    double2* hk = MG_DEVF(H.dr, double2, Hk);
    MG_CUDA_TRY(cudaMemcpy(hk, colmaj.data(), colmaj.size() * sizeof(double2), cudaMemcpyHostToDevice));
    ks_load_dense(H.pls, hk, nullptr, k, 0.0, s);
    launch_convert<double, float>(H.c32.W, H.c64.W, (long)(k + 1) * n2, Gate{}, s);
    MG_LAUNCH_CHECK();
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    H.defl_k = k;
    for (mg_handle_s* c : H.contexts) c->h.defl_k = k;
    return MG_OK;
}

mg_status mg_coarse_solve(mg_handle h, int precision, int nrhs, const void* b, void* x, double tol, int flags,
                          long long spin, void* stream, long long* iters, int* converged, mg_coarse_info* info) {
    if (!h || !b || !x) return set_error("handle, b and x must be non-NULL"), MG_EINVAL;
    Handle& H = h->h;
    if (H.is_context) return set_error("call mg_coarse_solve on the hierarchy owner"), MG_EINVAL;
    if (H.defl_k == 0) return set_error("no deflation space: solve once or call mg_set_deflation"), MG_EINVAL;
    if (!(tol > 0.0 && tol < 1.0)) return set_error("tol must be in (0, 1)"), MG_EINVAL;
    if (spin < 0) return set_error("spin must be >= 0"), MG_EINVAL;
    if (flags & ~MG_COARSE_PROBE_TIMEOUT) return set_error("unknown flags %d", flags), MG_EINVAL;
    if (precision == MG_BF16 || precision == MG_F16) {  // the batched tensor-core solve
        if (nrhs < 1 || nrhs > 64) return set_error("nrhs must be in [1, 64]"), MG_EINVAL;
        MG_TRY(device_vectors(b, "b"));
        MG_TRY(device_vectors(x, "x"));
        std::vector<long long> it(nrhs, 0);
        const mg_status st = coarse_solve_block(H, static_cast<const float2*>(b), static_cast<float2*>(x), nrhs, tol,
                                                precision == MG_F16, static_cast<cudaStream_t>(stream), it.data(),
                                                (flags & MG_COARSE_PROBE_TIMEOUT) != 0, (long)spin);
        if (st != MG_OK && st != MG_ETIMEOUT) return st;
        for (int r = 0; r < nrhs; ++r) {
            if (iters) iters[r] = it[r];
            if (converged) converged[r] = it[r] < (long long)H.p.proj_max_cycles * std::max(H.p.dr_m - H.defl_k, 1);
        }
        if (info) {
            *info = mg_coarse_info{};
            info->timeouts = st == MG_ETIMEOUT ? 1 : 0;
        }
        return st;
    }
    if (precision != MG_F64 && precision != MG_F32) return set_error("unknown precision %d", precision), MG_EINVAL;
    if (nrhs < 1 || nrhs > 2 || (nrhs == 2 && precision != MG_F32))
        return set_error("nrhs must be 1, or 2 (the paired kernel) with MG_F32"), MG_EINVAL;
    if (nrhs == 2 && flags) return set_error("the timeout probe is built into the single kernel only"), MG_EINVAL;
    MG_TRY(device_vectors(b, "b"));
    MG_TRY(device_vectors(x, "x"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long n2 = H.L64[2].n;
    Handle* HH[2] = {&H, nullptr};
    if (nrhs == 2) {  // the second right-hand side runs on a solve context's workspaces
        if (H.contexts.empty()) {
            mg_handle_s* c = nullptr;
            MG_TRY(make_solve_context(h, &c));
            H.contexts.push_back(c);
        }
        HH[1] = &H.contexts[0]->h;
        HH[1]->defl_k = H.defl_k;
    }
    for (int r = 0; r < nrhs; ++r) MG_CUDA_TRY(cudaMemsetAsync(HH[r]->cstats, 0, sizeof(CoopStats), s));
    if (precision == MG_F64) {
        CoopArgs<double> a = coarse_args<double>(H, static_cast<const double2*>(b), static_cast<double2*>(x), H.c64.r,
                                                 H.c64.V, H.cpart, H.cpart_ctas, H.cstats, tol);
        a.spin = spin;
        a.probe = (flags & MG_COARSE_PROBE_TIMEOUT) ? 1 : 0;
        MG_TRY(launch_coarse_proj<double>(a, s));
    } else {
        const float2* bf = static_cast<const float2*>(b);
        float2* xf = static_cast<float2*>(x);
        CoopArgs<float> a[2];
        for (int r = 0; r < nrhs; ++r) {
            Handle& C = *HH[r];
            a[r] = coarse_args<float>(C, bf + (long)r * n2, xf + (long)r * n2, C.c32.r, C.c32.V, C.cpart,
                                      C.cpart_ctas, C.cstats, tol);
            a[r].spin = spin;
            a[r].probe = (flags & MG_COARSE_PROBE_TIMEOUT) ? 1 : 0;
        }
        if (nrhs == 2) {
            bool launched = false;
            MG_TRY(launch_coarse_proj_pair(a[0], a[1], s, &launched));
            if (!launched) return set_error("the paired coarse kernel does not fit this coarse grid"), MG_EINVAL;
        } else {
            MG_TRY(launch_coarse_proj<float>(a[0], s));
        }
    }
    MG_LAUNCH_CHECK();
    long long timeouts = 0;
    CoopStats cs[2]{};
    for (int r = 0; r < nrhs; ++r) {
        MG_CUDA_TRY(cudaMemcpyAsync(H.pinned, HH[r]->cstats, sizeof(CoopStats), cudaMemcpyDeviceToHost, s));
        MG_CUDA_TRY(cudaStreamSynchronize(s));
        std::memcpy(&cs[r], H.pinned, sizeof(CoopStats));
        if (iters) iters[r] = cs[r].iters;
        if (converged) converged[r] = cs[r].unconverged == 0 ? 1 : 0;
        timeouts += cs[r].timeouts;
    }
    if (info) {
        info->ctas = cs[0].ctas;
        info->sites_per_cta = cs[0].spc;
        info->dataflow = cs[0].flow;
        info->dcgs2 = cs[0].dc;
        info->half_operator = cs[0].half;
        info->shared_blocks = cs[0].ash;
        info->paired = cs[0].paired;
        info->tensor_apply = cs[0].mma;
        info->cycles = cs[0].cycles;
        info->timeouts = timeouts;
    }
    if (timeouts) return set_error("coarse solve: a bounded wait of the dataflow exchange gave up"), MG_ETIMEOUT;
    return MG_OK;
}

mg_status mg_apply_block(mg_handle h, int level, int precision, int nrhs, const void* x, void* y, void* stream) {
    if (!h || !x || !y || x == y) return set_error("handle, x and y must be distinct non-NULL pointers"), MG_EINVAL;
    if (level < 1 || level > 2) return set_error("level must be 1 or 2"), MG_EINVAL;
    if (precision != MG_BF16 && precision != MG_F16) return set_error("precision must be MG_BF16 or MG_F16"), MG_EINVAL;
    if (nrhs < 8 || nrhs > 64 || nrhs % 8) return set_error("nrhs must be a multiple of 8 in [8, 64]"), MG_EINVAL;
    MG_TRY(device_vectors(x, "x"));
    MG_TRY(device_vectors(y, "y"));
    return apply_block(h->h, level, static_cast<const float2*>(x), static_cast<float2*>(y), nrhs, precision == MG_F16,
                       static_cast<cudaStream_t>(stream));
}

}  // extern "C"
