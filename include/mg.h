/*
 * mg.h - C ABI of the GB300 deflated multigrid solver for the 2D Schwinger-model
 * Wilson-Dirac operator (Whyte, Wilcox, Morgan, "Deflated GMRES with Multigrid
 * for Lattice QCD", arXiv:1912.02868).
 *
 * The library solves D x = b for many right-hand sides b with one operator D
 * (Section 2: FGMRES(8) outer solver; three-grid adaptive multigrid V-cycle with
 * GMRES(2) pre/post smoothing on the fine and intermediate grids; GMRES-DR(m,k)
 * on the coarsest grid at the first outer iteration and GMRES-Proj(m,k) at every
 * later one and for every later right-hand side).
 *
 * Conventions for every entry point
 *  - Complex numbers are interleaved (re, im): complex128 = 2 doubles,
 *    complex64 = 2 floats.
 *  - Gauge field: complex128[L_t][L_x][2], mu = 0 is the x link, mu = 1 the t link,
 *    |U| = 1.  The fermion is periodic in x and antiperiodic in t.
 *  - Fine spinor: complex[L_t][L_x][2] (site = x + L_x t, spin fastest).
 *  - Coarse vector on a grid of N_t x N_x sites: complex[N_t][N_x][24], dof
 *    k = 12 c + j (chirality c, near-null vector j).
 *  - Pointers marked "host or device" may point to pageable host memory, pinned
 *    host memory or device memory of the current device; the library tells them
 *    apart with cudaPointerGetAttributes.  Pointers marked "device" must be
 *    device memory.  The caller keeps ownership of every pointer it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is ordered on that stream and returns after the results it
 *    reports on the host are complete.
 *  - Errors come back only as status codes; mg_last_error() returns a message
 *    for the calling thread's last failure.  No entry point aborts the process.
 *  - Handles are not thread-safe: one thread at a time per handle.
 */
#ifndef MG_H
#define MG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_handle_s* mg_handle;

typedef enum {
    MG_OK = 0,
    MG_EINVAL = -1,     /* invalid argument (shape, pointer, parameter) */
    MG_ENOMEM = -2,     /* device allocation failed */
    MG_ECUDA = -3,      /* a CUDA runtime call failed */
    MG_ENOTCONV = -4,   /* a solve reached its iteration limit */
    MG_EBUDGET = -5,    /* reserved for memory-budget admission */
    MG_ETIMEOUT = -6    /* a bounded device wait gave up (the coarse kernel's dataflow exchange) */
} mg_status;

/* coarsest-grid solver (Section 2) */
enum { MG_COARSE_DR_PROJ = 0, /* GMRES-DR(m,k) first, then GMRES-Proj(m,k) */
       MG_COARSE_CGNE = 1     /* CGNE to coarse_tol_rest at every outer iteration */ };

/* arithmetic of the preconditioner; the outer FGMRES is always FP64 */
enum { MG_FP64 = 0,        /* everything in FP64 */
       MG_MIXED = 1,       /* V-cycle in FP32; deflation space built in FP64 */
       MG_MIXED_BF16 = 2,  /* block solve: right-hand sides in lockstep blocks of rhs_block, V-cycle
                              in FP32 with the intermediate and coarsest 24x24 block products on
                              tensor cores (BF16 operator, FP32 vectors split into two BF16 parts,
                              FP32 accumulation); deflation space built in FP64 */
       MG_MIXED_FP16 = 3   /* the same with an FP16 operator */ };

typedef struct {
    int levels;            /* grids in the hierarchy: 3 */
    int block;             /* blocking per direction: 4 (4^2 blocks) */
    int nvec;              /* near-null vectors per level: 12 */
    int smooth_steps;      /* GMRES steps of each smoother: 2 */
    int fgmres_m;          /* outer restart length: 8 */
    int max_outer;         /* outer iteration limit per right-hand side */
    int coarse_solver;     /* MG_COARSE_DR_PROJ or MG_COARSE_CGNE */
    int dr_m, dr_k;        /* GMRES-DR / GMRES-Proj (m, k): 30, 10 */
    int dr_max_cycles;     /* GMRES-DR cycle limit (100) */
    int dr_stall_cycles;   /* GMRES-DR ends after this many cycles without progress (2) */
    int proj_max_cycles;   /* GMRES-Proj cycle limit per solve (1000) */
    int cgne_max_iters;    /* CGNE iteration limit per solve */
    int nullvec_max_iters; /* CG iteration limit of each near-null solve */
    double nullvec_tol;    /* near-null solve tolerance: 1e-4 */
    double coarse_tol_first; /* GMRES-DR tolerance of the first coarse solve */
    double coarse_tol_rest;  /* GMRES-Proj / CGNE tolerance: 1e-8 */
    int precision;         /* MG_FP64 or MG_MIXED */
    unsigned long long seed; /* start vectors of the near-null solves when none are given */
    int method;            /* MG_METHOD_MG (default) or MG_METHOD_FINE_DEFLATION */
    int parallel;          /* right-hand sides of one mg_solve solved concurrently (1):
                              with > 1, the first right-hand side of a handle builds the
                              deflation space alone, then up to `parallel` solve contexts
                              (shared hierarchy, own workspaces and streams) share the rest */
    double partial_tol;    /* 0 (default): V-cycle.  > 0: partial intermediate solve (Section 2
                              variant): the intermediate system is solved to this relative
                              residual (the paper: 0.2) by FGMRES(fgmres_m) preconditioned
                              with the two-grid cycle; coarse solves then go to coarse_tol_rest
                              within a right-hand side's first outer iteration (GMRES-DR
                              first) and to coarse_tol_partial after it */
    double coarse_tol_partial; /* coarse tolerance after the first outer iteration in the
                                  partial mode: 1e-2 */
    int partial_max_iters; /* FGMRES iteration limit of one partial intermediate solve (200) */
    int pair_rhs;          /* 1: with parallel > 1, each concurrent worker solves two right-hand
                              sides in lockstep on two contexts, and their coarsest solves run as
                              one cluster kernel that streams the coarse operator once for both
                              (mixed precision, V-cycle, deflated coarse solve, device buffers;
                              the paired kernel applies with FP32 FMAs, and the results equal
                              those of separate solves with coarse_mma = 0).  0 (default): one
                              right-hand side per worker */
    int vcycle_graph;      /* 1 (default): in mixed precision, once the deflation space exists, the
                              V-cycle (grid-0 and grid-1 smoothing and transfers, the coarse
                              GMRES-Proj kernel) is captured into a CUDA graph and replayed: one
                              launch a V-cycle, the same kernels and arguments.  Not with the
                              partial intermediate solve or with apply timing on.  0: launched
                              kernel by kernel */
    int coarse_half;       /* 1 (default): in mixed precision, the coarsest operator streamed by the
                              GMRES-Proj cluster kernels each Arnoldi step is an FP16 copy (each
                              part rounded once from FP64), multiplied in FP32; the deflation build
                              (GMRES-DR) keeps the FP64 operator.  0: the FP32 copy */
    int coarse_dcgs2;      /* 1: the single-right-hand-side GMRES-Proj cluster kernel orthogonalises
                              by delayed CGS2, one exchange per Arnoldi step instead of two (when
                              its basis and staging sit in shared memory; the paired kernel keeps
                              CGS2).  0 (default): CGS2 */
    int rhs_block;         /* MG_MIXED_BF16 / MG_MIXED_FP16: right-hand sides solved in lockstep per
                              block, 1..64 (64).  Each has its own FGMRES(fgmres_m) in FP64 and
                              converges on its own true residual; the V-cycle and the coarse
                              GMRES-Proj solves of a block run batched (the first right-hand side
                              of a handle builds the deflation space alone first).  The outer
                              iteration limit max_outer is checked at restarts */
    int lowrank_hops;      /* 1 (default): the intermediate grid's four hop blocks of every site
                              applied as rank-4 factors Q R (each block of P^+ D P sums four
                              boundary-site terms, each with a rank-1 spin projector), the same
                              operator to rounding, with about half the bytes and FP64 work of the
                              dense blocks; 0: dense blocks.  The factors come from a pivoted
                              Gram-Schmidt of each dense block at set-up; a block whose rank-4
                              reconstruction errs by more than 1e-11 relative keeps the handle
                              dense (mg_solve_stats is unaffected) */
    int autotune;          /* 1 (default): at set-up, each level apply (the fine Wilson-Dirac
                              apply; the FP32 block stencils of grids 1 and 2) is timed with every
                              candidate launch shape and the fastest kept (mg_launch_shape).  A
                              shape only groups sites into blocks (for the fine apply: threads per
                              block, tiles staged in shared memory, or columns of sites a thread),
                              so results are the same bit for bit with any choice.  0: the built-in shapes */
    int coarse_mma;        /* 1 (default): with coarse_half, the single-right-hand-side GMRES-Proj
                              cluster kernel applies the FP16 operator on tensor cores (mma.sync
                              m16n8k16, FP32 accumulation) to each basis vector split into two
                              FP16 parts (22 bits), where it holds the blocks of three directions
                              in shared memory and runs CGS2 in dataflow mode (the 256^2 lattice's
                              16^2 x 24 coarse grid and smaller); elsewhere, and with 0, FP32 FMAs */
} mg_params;

/* solver of mg_solve (Section 2 compares both) */
enum { MG_METHOD_MG = 0,             /* FGMRES(8) preconditioned by the deflated V-cycle */
       MG_METHOD_FINE_DEFLATION = 1, /* no multigrid: GMRES-DR(m,k) on the fine operator for the
                                        first right-hand side, GMRES-Proj(m,k) afterwards, FP64;
                                        mg_solve's iters then counts Krylov steps */
       MG_METHOD_FINE_CGNE = 2       /* no multigrid: CGNE on the fine operator (CG on D D^+ y = b,
                                        x = D^+ y) to the tolerance, limit cgne_max_iters, FP64;
                                        iters counts CG steps (2 applies each) */ };

typedef struct {
    long long mvps[3];       /* operator applications per grid (fine, intermediate, coarse) */
    double fine_equiv_mvps;  /* Section 3, Eq. 1: fine + (n1/n0) int + (n2/n0) coarse */
    int outer_iters;         /* FGMRES iterations summed over the right-hand sides */
    int coarse_solves;       /* coarsest-grid solves */
    long long coarse_iters;  /* Krylov iterations of all coarsest-grid solves */
    int dr_solves;           /* coarse solves done by GMRES-DR (builds the deflation space) */
} mg_solve_stats;

/* Fill *p with the defaults listed beside each field. */
mg_status mg_default_params(mg_params* p);

/*
 * Build the three-grid hierarchy of D(m0) on an L_x x L_t lattice (Section 2,
 * first paragraph): 12 near-null vectors from D D^+ e = -D D^+ x solved by CG to
 * nullvec_tol with psi = x + e, global orthonormalisation, chiral doubling,
 * local block x block orthonormalisation into P, D^ = P^+ D P, all repeated on
 * D^ for the coarsest grid.
 *   gauge    host or device, complex128[L_t][L_x][2] (copied; not kept)
 *   L_x, L_t multiples of block^2 (= 16)
 *   nvec     12 (the only value built); block 4
 *   p        parameters (NULL = defaults)
 *   starts0  host or device, complex128[nvec][L_t][L_x][2]: the random x of the
 *            fine near-null solves; NULL = generated from p->seed
 *   starts1  host or device, complex128[nvec][L_t/4][L_x/4][24] for the
 *            intermediate grid; NULL = generated from p->seed
 *   out      receives the handle; release it with mg_destroy
 * Errors: MG_EINVAL (shape, parameters, rank-deficient local block),
 *         MG_ENOMEM, MG_ECUDA.
 */
mg_status mg_setup(const void* gauge, int L_x, int L_t, double m0, int nvec, int block,
                   const mg_params* p, const void* starts0, const void* starts1,
                   void* stream, mg_handle* out);

/*
 * Same hierarchy, but from given near-null vectors psi (the result of step 1 of
 * the set-up) instead of solving for them: used to compare the set-up and the
 * solve with an independent implementation on identical prolongators.
 *   nullvecs0 host or device, complex128[nvec][L_t][L_x][2]
 *   nullvecs1 host or device, complex128[nvec][L_t/4][L_x/4][24]
 */
mg_status mg_setup_from_vectors(const void* gauge, int L_x, int L_t, double m0, int nvec, int block,
                                const mg_params* p, const void* nullvecs0, const void* nullvecs1,
                                void* stream, mg_handle* out);

/*
 * Solve D x_i = b_i, i < nrhs, to true relative residual ||b - D x|| / ||b|| <= tol,
 * recomputed in FP64 (Section 2: FGMRES(8) preconditioned by the V-cycle).
 *   b        host or device, complex128[nrhs][L_t][L_x][2]
 *   x        host or device, same shape; output (the initial guess is zero)
 *   iters    host int[nrhs] or NULL: outer iterations per right-hand side
 *   relres   host double[nrhs] or NULL: final true relative residuals
 *   stats    host or NULL: counters summed over this call
 * The coarse deflation space is built by the first coarse solve of the handle's
 * first solve and kept for all later outer iterations and right-hand sides.
 * Returns MG_ENOTCONV when some right-hand side hit max_outer; x then holds the
 * last iterate and relres its true residual.
 */
mg_status mg_solve(mg_handle h, const void* b, void* x, int nrhs, double tol, void* stream,
                   int* iters, double* relres, mg_solve_stats* stats);

/* Forget the deflation space (coarse, or fine for MG_METHOD_FINE_DEFLATION):
 * the next solve runs GMRES-DR again. */
mg_status mg_reset_deflation(mg_handle h);

/* Release every device buffer of the handle. NULL is accepted. */
mg_status mg_destroy(mg_handle h);

/* Message of the calling thread's last failed call ("" if none). */
const char* mg_last_error(void);

/* ------------------------------------------------------------------------- */
/* Operator-level entry points (one kernel each), for parity checks and for  */
/* callers that build their own solvers on the hierarchy.                    */
/* ------------------------------------------------------------------------- */

/* precision of the operator-level calls: the vectors are complex128 for
 * MG_F64 and complex64 for MG_F32, MG_BF16 and MG_F16; MG_BF16 / MG_F16 are the
 * tensor-core block products (BF16 / FP16 operator, FP32 vectors, FP32 accumulation) */
enum { MG_F64 = 0, MG_F32 = 1, MG_BF16 = 2, MG_F16 = 3 };

/*
 * y_r = D^ x_r, r < nrhs, on grid `level` (1 or 2) with the tensor-core block
 * stencil of the block solve (Section 2's Galerkin operator D^ = P^+ D P, 24x24
 * complex blocks as real 48x48 products in mma.sync m16n8k16 tiles).
 *   precision  MG_BF16 or MG_F16: the operator rounded once from FP64
 *   nrhs       a multiple of 8 (eight right-hand sides share an MMA tile), <= 64
 *   x, y       device, complex64[nrhs][n_level] (must not alias)
 */
mg_status mg_apply_block(mg_handle h, int level, int precision, int nrhs, const void* x, void* y, void* stream);

/*
 * y = D x (dagger = 0) or y = D^+ x = sigma_3 D sigma_3 x (dagger = 1) on one
 * grid of the hierarchy: level 0 is the Wilson-Dirac operator (Section 2), levels
 * 1 and 2 the Galerkin stencils D^ = P^+ D P with D^+ = sigma3^ D^ sigma3^.
 *   x, y  device, complex[n_level] in the precision given (must not alias)
 */
mg_status mg_apply(mg_handle h, int level, int dagger, int precision, const void* x, void* y, void* stream);

/* y_c = P^+ y (restriction from `level` to level+1), Section 2. device pointers. */
mg_status mg_restrict(mg_handle h, int level, int precision, const void* fine, void* coarse, void* stream);

/* y = P y_c (prolongation from level+1 to `level`), Section 2. device pointers. */
mg_status mg_prolong(mg_handle h, int level, int precision, const void* coarse, void* fine, void* stream);

/*
 * Copy out the hierarchy (host or device destination, complex128):
 *   mg_get_stencil: level 1 or 2, complex128[N_t][N_x][5][24][24], directions
 *     (self, +x, -x, +t, -t), entry [k][l] maps dof l of the neighbour to dof k.
 *   mg_get_prolongator: level 0 or 1, complex128[B_t][B_x][2][12][16][h],
 *     h = 1 (level 0) or 12 (level 1); see the layout of P in the set-up.
 *   mg_get_deflation: W complex128[k+1][n_2] and H complex128[k+1][k]
 *     (row-major), with D W_k = W H; *k_out = k (0 before the first coarse solve).
 *     Either pointer may be NULL to query k only.
 */
mg_status mg_get_stencil(mg_handle h, int level, void* out);
mg_status mg_get_prolongator(mg_handle h, int level, void* out);
mg_status mg_get_deflation(mg_handle h, void* W, void* H, int* k_out);

/*
 * Replace the handle's coarse deflation space (Section 2: the space (V_{k+1}, H_k)
 * that GMRES-DR leaves for the GMRES-Proj solves) with a given one:
 *   W   host or device, complex128[k+1][n_2], orthonormal rows
 *   H   host or device, complex128[k+1][k] (row-major), D^ W_k = W H
 *   k   1 <= k <= dr_m
 * Every later coarse solve of the handle (and of its solve contexts) is then a
 * GMRES-Proj solve with this space.  Used to run the coarse solves of the
 * library and of an independent implementation on the same space.
 * Errors: MG_EINVAL (sizes, a solve context), MG_ECUDA.
 */
mg_status mg_set_deflation(mg_handle h, const void* W, const void* H, int k);

/* flags of mg_coarse_solve */
enum { MG_COARSE_PROBE_TIMEOUT = 1 };

/* launch shape of the last mg_coarse_solve */
typedef struct {
    int ctas;            /* CTAs of the cluster */
    int sites_per_cta;   /* coarse sites each CTA owns */
    int dataflow;        /* 1: st.async / byte-counted mbarrier exchange in each Arnoldi step */
    int dcgs2;           /* 1: delayed CGS2 ran (one exchange per step) */
    int half_operator;   /* 1: the FP16 copy of the operator was streamed */
    int shared_blocks;   /* 1: the FP16 blocks of three directions were held in shared memory */
    int paired;          /* 1: the two-right-hand-side kernel */
    long long cycles;    /* GMRES cycles of right-hand side 0 */
    long long timeouts;  /* CTAs in which a bounded wait gave up */
    int tensor_apply;    /* 1: the apply ran on tensor cores (mg_params.coarse_mma) */
} mg_coarse_info;

/*
 * One projected solve of the coarsest system D^ x = b (Section 2: GMRES-Proj(m,k)
 * with the handle's deflation space, from x = 0, until the least-squares
 * residual estimate is <= tol ||b||), run by the same kernels, with the same
 * launch shape, as the coarse solves inside the V-cycle.
 *   precision  MG_F64: complex128 vectors and the FP64 operator; MG_F32:
 *              complex64 vectors (the FP16 operator copy when coarse_half,
 *              delayed CGS2 when coarse_dcgs2); MG_BF16 / MG_F16: the batched
 *              GMRES-Proj of the block solve, complex64 vectors, tensor-core
 *              applies (info reports ctas = 0)
 *   nrhs       1, or 2 with MG_F32 (the two-right-hand-side kernel), or 1..64
 *              with MG_BF16 / MG_F16
 *   b, x       device, [nrhs][n_2] in that precision; x is output
 *   flags      MG_COARSE_PROBE_TIMEOUT (tests): before the first cycle every CTA
 *              waits, bounded by `spin`, on a barrier that nothing completes, so
 *              the give-up path runs; the call then returns MG_ETIMEOUT and the
 *              handle stays usable.  MG_BF16 / MG_F16: every CTA of the batched
 *              cycle kernel waits so at the start of each cycle (info->timeouts
 *              = 1); the probe needs the cycle kernel's resident grid (MG_EINVAL
 *              on coarse grids that run the three-kernel steps)
 *   spin       try_wait rounds (MG_BF16 / MG_F16: tile-barrier polls) before a
 *              bounded wait gives up (0: 2^20; 2^18 polls)
 *   iters      host long long[nrhs] or NULL: Krylov steps per right-hand side
 *   converged  host int[nrhs] or NULL
 *   info       host or NULL: the launch shape
 * Needs a deflation space (a first mg_solve, or mg_set_deflation).
 * Errors: MG_EINVAL, MG_ECUDA, MG_ETIMEOUT (a bounded wait gave up).
 */
mg_status mg_coarse_solve(mg_handle h, int precision, int nrhs, const void* b, void* x, double tol, int flags,
                          long long spin, void* stream, long long* iters, int* converged, mg_coarse_info* info);

/* Grid sizes: sites per direction and dofs per site of `level`. */
mg_status mg_level_shape(mg_handle h, int level, int* n_x, int* n_t, int* dof);

/* How `level` (1 or 2) applies its stencil: *factored = 1 when its hop blocks run as
 * rank-4 factors (lowrank_hops, intermediate grid only), and *max_rel_err (host or
 * NULL) the largest relative Frobenius error of those factors against the dense
 * blocks (0 when not factored). */
mg_status mg_stencil_info(mg_handle h, int level, int* factored, double* max_rel_err);

/* Launch shape of the apply of `level` (0..2) in `precision` (MG_F64 or MG_F32), as
 * the set-up's autotuner chose it (mg_params.autotune): *shape = 0 for the built-in
 * shape, else threads per block of the one-thread-per-site kernel, 1000 + r for
 * tiles of 32 x r sites staged in shared memory, or 2000 + r for columns of r sites
 * a thread with the x neighbours taken from adjacent lanes (level 0), or sites per
 * block (FP32 stencils of levels 1 and 2).  us (host, double[2], or NULL): the time of one apply with the
 * chosen and with the built-in shape, in microseconds, as timed at set-up on this
 * GPU (0 where nothing was tuned: FP64 stencils, autotune off).  The shape never
 * changes results: it only groups sites into blocks. */
mg_status mg_launch_shape(mg_handle h, int level, int precision, int* shape, double* us);

/* Pin the launch shape of the apply of `level` in `precision`: 0 (built-in), or one
 * of the candidates the autotuner tries: 64, 128, 256 threads per block, 1004 and
 * 1008 (tiles of 32 x 4 and 32 x 8 sites whose spinors, with a one-site halo, and
 * links are staged in shared memory), or 2002 and 2004 (each thread keeps a column
 * of 2 or 4 sites along t in registers and takes its x neighbours from the adjacent
 * lanes of its warp) at level 0;
 * 4, 8, 12, 16 sites per block for the FP32 stencil with rank-4 hop factors; 4, 8,
 * 16, 24, 32 for the dense FP32 stencil.  The FP64 stencils take 0 only.  A captured
 * V-cycle graph of the handle is dropped and captured again; solve contexts made
 * afterwards copy the shape.  MG_EINVAL for any other shape. */
mg_status mg_set_launch_shape(mg_handle h, int level, int precision, int shape);

/*
 * Standalone Wilson-Dirac apply without a hierarchy (Section 2):
 *   gauge  device, complex128[L_t][L_x][2] (MG_F64) or complex64 (MG_F32)
 *   x, y   device, complex[L_t][L_x][2]; y = D(m0) x or D^+ x
 */
mg_status mg_wilson_apply(const void* gauge, int L_x, int L_t, double m0, int dagger, int precision,
                          const void* x, void* y, void* stream);

/* ------------------------------------------------------------------------- */
/* Serving: continuous batching of solve requests over many operators        */
/* (the serving pattern layered on the method; the paper has no serving).    */
/* ------------------------------------------------------------------------- */

typedef struct mg_server_s* mg_server;

typedef struct {
    unsigned long long key;   /* caller's name of the operator (gauge field, m0, lattice) */
    const void* gauge;        /* host or device, complex128[L_t][L_x][2]; read only when
                                 `key` is not resident; valid until the request completes */
    int L_x, L_t;
    double m0;
    const void* starts0;      /* optional near-null start vectors as in mg_setup (NULL: seed) */
    const void* starts1;
    const void* b;            /* host or device, complex128[nrhs][L_t][L_x][2] */
    void* x;                  /* host or device, same shape; output */
    int nrhs;                 /* >= 1 */
    double tol;               /* true relative residual per right-hand side */
} mg_request;

typedef struct {
    int resident_keys;              /* operators whose hierarchy is in HBM */
    unsigned long long device_bytes;/* device bytes held by resident hierarchies and contexts */
    long long evictions;            /* hierarchies dropped to admit others */
    long long cold_starts;          /* hierarchies built */
    long long completed;            /* requests finished */
    long long queued_items;         /* right-hand sides waiting for a worker */
    long long batches;              /* solve calls run by the workers */
    int max_batch;                  /* most right-hand sides solved together in one call */
    unsigned long long demand_bytes;/* estimated device bytes of all keys ever requested, i.e.
                                       what keeping every one of them resident would take */
} mg_server_info;

/*
 * Create a server with `workers` host threads on the current device.  Every
 * right-hand side of every request is one work item; items run in arrival order
 * on solve contexts (own workspaces and CUDA stream) of their key's hierarchy,
 * so requests of different keys and lattice sizes overlap on the GPU and new
 * requests join as soon as a worker is free.  A key's hierarchy is built on its
 * first request (mg_setup with `p`), and its coarse deflation space by one solve
 * of a fixed seeded right-hand side, so results do not depend on which requests
 * came first.  Hierarchies stay resident (LRU) while the estimated device bytes
 * stay within hbm_budget_bytes (0 = unlimited); a new key waits until an idle
 * hierarchy can be evicted.
 * With p->precision MG_MIXED_BF16 or MG_MIXED_FP16 a key runs one lockstep block
 * solve at a time on its hierarchy (no solve contexts): the worker that takes
 * an item also takes every queued item of the same key and tolerance, from any
 * request, up to p->rhs_block, and solves them together with tensor-core block
 * products; items that arrive meanwhile join the next block.  A block gathered
 * from several requests is staged in a device buffer of the worker (counted in
 * device_bytes).  Results then depend on the block they ran in only through
 * rounding: each meets its tolerance either way.
 */
mg_status mg_server_create(const mg_params* p, unsigned long long hbm_budget_bytes, int workers,
                           mg_server* out);
/* Queue a request; *ticket identifies it for mg_server_wait. */
mg_status mg_server_submit(mg_server s, const mg_request* r, unsigned long long* ticket);
/* Block until the request is done.  iters/relres: host [nrhs] or NULL;
 * latency_s: host or NULL, seconds from submission to completion. */
mg_status mg_server_wait(mg_server s, unsigned long long ticket, int* iters, double* relres,
                         double* latency_s);
/* Non-blocking mg_server_wait: *done = 0 and MG_OK while the request is still
 * running (the ticket stays valid); once it has finished, *done = 1, the
 * outputs and the status are those of mg_server_wait, and the ticket is
 * released. */
mg_status mg_server_poll(mg_server s, unsigned long long ticket, int* done, int* iters, double* relres,
                         double* latency_s);
mg_status mg_server_stats(mg_server s, mg_server_info* out);
/* Stop the workers (queued items are dropped) and free every hierarchy. */
mg_status mg_server_destroy(mg_server s);

/* ------------------------------------------------------------------------- */
/* Instrumentation                                                           */
/* ------------------------------------------------------------------------- */

/*
 * Time every operator apply on grid `level` of the handle with CUDA events on
 * the stream the apply runs on (enable = 1), or stop (enable = 0).  Enabling
 * resets the totals.  mg_timing_read waits for the last recorded event and
 * returns the summed apply time in milliseconds and the number of applies.
 * Meant for roofline reports; the events add a few microseconds of host work
 * per apply.  On the coarsest grid (level 2) the timed unit is one whole
 * projected coarse solve (a single kernel); applies inside GMRES-DR or CGNE
 * coarse solves are timed individually and may include steps skipped on the
 * device after convergence.
 */
mg_status mg_timing_enable(mg_handle h, int level, int enable);
mg_status mg_timing_read(mg_handle h, int level, double* total_ms, long long* launches);

/* Number of kernels this library has launched in this process so far. */
unsigned long long mg_kernel_launches(void);

/*
 * Allocation-free true residual (the paper has no counterpart: it is a
 * service for callers that may not allocate device memory, e.g. an
 * application whose pool owns all of HBM, or a thread that must not let
 * cudaMalloc/cudaFree synchronise the device while other streams run).
 * Computes r = b - D(m0) x with the solver's FP64 residual kernel and
 *   norms[0] = ||b - D x||_2,  norms[1] = ||b||_2.
 *   gauge     device, complex128[L_t][L_x][2] (caller-owned, read only)
 *   b, x      device, complex128[L_t][L_x][2] (read only)
 *   r         device, complex128[L_t][L_x][2] (written; must not alias b or x)
 *   norms     host, double[2] (written; the call waits for `stream`)
 * All four device pointers must be memory of the current device (MG_EINVAL
 * otherwise).  No device memory is allocated: the reductions use a fixed
 * 32 800-byte array in the library's device image, which bounds the lattice to at most 2^20 sites
 * (1024 x 1024); larger lattices return MG_EINVAL.  The first call on each
 * device looks up that array's address, so it should come before any stream
 * capture begins on the device.  There is one such array per device: calls
 * that can overlap on the GPU (other streams or host threads) race on it and
 * must be serialised by the caller.
 */
mg_status mg_wilson_residual_noalloc(const void* gauge, int L_x, int L_t, double m0, const void* b, const void* x,
                                     void* r, double* norms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
