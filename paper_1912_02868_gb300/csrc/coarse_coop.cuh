// Cooperative persistent kernel of the coarsest-grid GMRES-Proj solve.
#pragma once
#include "kstate.cuh"

namespace mg {

constexpr int MSMAX = 24;  // longest GMRES cycle of a projected solve (m - k): (30,10) -> 20, (40,16) -> 24
constexpr int PSTR = 64;   // stride of one CTA's partial sums

// device-side counters of the projected coarse solves
struct CoopStats {
    long long iters, cycles, solves, unconverged;
    long long timeouts;  // CTAs in which a bounded wait of the dataflow exchange gave up
    // shape of the last launch (written by its CTA 0): cluster size, coarse
    // sites per CTA, dataflow exchange, delayed CGS2, FP16 blocks in shared
    // memory, FP16 operator stream, two-right-hand-side kernel, tensor-core apply
    int ctas, spc, flow, dc, ash, half, paired, mma;
};

template <typename T>
struct CoopArgs {
    const C2<T>* A;    // coarse stencil, column-major 24x24 blocks
    const unsigned* Ah;  // or null: the same stencil in FP16 (real part in the low half), read
                         // instead of A by the push-mode apply (FP32 arithmetic)
    int Nx, Nt;        // coarse grid
    const C2<T>* f;    // right-hand side
    C2<T>* x;          // solution (output, initial guess zero)
    C2<T>* r;          // residual workspace
    C2<T>* V;          // Krylov basis, (ms + 1) rows of n
    const C2<T>* W;    // deflation space V_{k+1}, (k + 1) rows of n
    const KState* pls; // H_k and its QR factorisation
    int k, ms;         // deflation size, GMRES cycle length
    double tol;        // stop when ||r|| <= tol ||f||
    int max_cycles;
    double2* part;     // partial sums: 2 x part_ctas x PSTR
    int part_ctas;
    CoopStats* out;
    int spc;           // sites per CTA (set by the launcher)
    int vs;            // 1: own basis rows kept in shared memory (set by the launcher)
    int lsw;           // 1: one extra warp runs the least-squares updates (set by the launcher)
    int ash;           // 1: the FP16 blocks of the first directions are kept in shared memory
                       // (set by the launcher)
    int dc;            // 1: delayed CGS2, one exchange per Arnoldi step (dataflow push mode)
    int flow;          // 1: push mode exchanges each step's values by st.async into byte-counted
                       // barriers instead of cluster barriers (set by the launcher)
    long spin;         // try_wait rounds before a dataflow wait gives up (0: the default, 2^20)
    int probe;         // 1 (tests): before the first cycle every row thread waits, bounded by
                       // `spin`, on a barrier that nothing completes, so the give-up path runs
    int mma;           // 1: the apply runs on tensor cores where the kernel can (FP32 dataflow mode
                       // with the FP16 blocks in shared memory, CGS2): FP16 operator times the
                       // vector split into two FP16 parts, FP32 accumulation
};

template <typename T>
mg_status launch_coarse_proj(const CoopArgs<T>& a, cudaStream_t s);

// The projected solves of two right-hand sides of one coarsest operator (same
// A, deflation space and parameters; own f, x, r, V and counters) in one
// cluster kernel, in lockstep: each block entry of A is loaded once for both
// vectors and the two share each step's exchanges.  FP32 only.  *launched is
// false (and nothing is enqueued) when the shape does not fit the kernel (both
// basis slices in shared memory); the caller then launches the two one by one.
mg_status launch_coarse_proj_pair(const CoopArgs<float>& a0, const CoopArgs<float>& a1, cudaStream_t s,
                                  bool* launched);

}  // namespace mg
