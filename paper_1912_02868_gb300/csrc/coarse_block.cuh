// Fused Arnoldi step of the batched coarse GMRES-Proj (coarse_block.cu).
#pragma once
#include "batch.cuh"
#include "coarse_coop.cuh"

namespace mg {

constexpr int CB_PB = 32;       // partial slots per right-hand side: basis products, norm in the last
constexpr int CB_MAXCH = 256;   // site chunks (the partials of a slot are adjacent, one per chunk)
constexpr int CB_THREADS = 256;
#ifndef CB_WPR_DEF
#define CB_WPR_DEF 1
#endif
constexpr int CB_WPR = CB_WPR_DEF;     // the cycle kernel's warps per right-hand side
constexpr int CB_COOP_THREADS = (NB_TILE * CB_WPR + 1) * 32;  // and one pushing warp
constexpr int CB_MAXSPC = 16;   // coarse sites per chunk of the step kernels (the cycle kernel sizes its own)

struct CBArgs {
    const unsigned* Af;  // coarsest operator in MMA fragment order (launch_pack_frag)
    int Nx, Nt;          // coarsest grid
    long n;              // entries of a vector (sites x 24)
    float2* V;           // basis rows V[i][r][n], i <= m - k
    long row;            // nbp * n: stride of one basis index
    KState* ks;          // [nbp] FP64 least squares of each right-hand side
    int* gbuf;           // [2][nbp] step gates by step parity
    float2* p1;          // [nbp][CB_PB][CB_MAXCH] partial sums of the first Gram pass
    float2* p2;          // the same for the second pass and the norm
    float2* h1;          // [nbp][CB_PB] reduced first-pass products
    float2* h2;          // [nbp][CB_PB] reduced second-pass products; slot CB_PB - 1: (h_{j+1,j}, 1 / h_{j+1,j})
    unsigned* ticket;    // [2][nbp / 8] arrivals of the chunks of a tile, per pass (step kernels)
    unsigned* bar;       // [nbp / 8][2] tile barrier (count, generation) of the cycle kernel, then
                         // one word that nothing writes (the probe's)
    int spc, nchunks, nbp;
    int coop;            // 1: geometry of the cycle kernel
    int probe;           // test probe: every CTA first waits (bounded) on the word nothing writes
};

// chunk size for nsite coarse sites and nbp right-hand sides (nbp % 8 == 0):
// for the step kernels, or (returning false when it cannot) for the cycle
// kernel, whose whole grid must be resident at once
void cb_geometry(CBArgs& a, long nsite, int nbp);
bool cb_geometry_cycle(CBArgs& a, long nsite, int nbp, bool fp16);
// gbuf[0][r] = ks[r].step_gate, gbuf[1][r] = -1 (after the cycle's start)
void launch_cb_gate_init(const CBArgs& a, cudaStream_t s);
// Arnoldi step jh of every right-hand side whose gate is open: v_{jh+1} and the
// least-squares column jh (three kernels; the tickets must be zero initially and
// are left zero)
void launch_cb_step(const CBArgs& a, int jh, bool fp16, cudaStream_t s);
// all ms steps of a cycle in one cooperative launch (cb_geometry_cycle); a tile
// barrier that waits longer than `spin` polls sets *err
mg_status launch_cb_cycle(const CBArgs& a, int ms, bool fp16, long spin, int* err, cudaStream_t s);

}  // namespace mg
