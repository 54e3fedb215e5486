// Batched forms of the flag pass and the two sweeps: one launch for all cases
// of a batch.  Each CTA takes its case's Params from the device table (row =
// step parity, step from the device counter) into shared memory and runs the
// single-lattice body on it.
#pragma once

#include "k_sweep.cuh"

namespace lbmmb {

// g_chain CTAs per case, persistent over that case's flag work list.
template <typename S, int Q>
__global__ void __launch_bounds__(BRICK) k_flags_batch(BatchArgs B) {
    __shared__ Params sP;
    __shared__ SmemParticles sp;
    __shared__ int s_next[2];
    const int c = blockIdx.x / B.g_chain, lb = blockIdx.x % B.g_chain;
    load_case_params(B, c, B.ctr, sP);
    flags_work<S, Q>(sP, sp, s_next, lb);
}

// g_chain CTAs per case over its near bricks; the last CTA of the launch
// advances the particle chain's step counter.
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, kNearCtasPerSm) k_sweep_near_batch(BatchArgs B) {
    __shared__ Params sP;
    __shared__ SmemParticles sp;
    __shared__ double red[BRICK / 32][6];
    __shared__ int s_links;
    __shared__ LinkScratch ls;
    __shared__ int s_next[2];
    const int c = blockIdx.x / B.g_chain;
    load_case_params(B, c, B.ctr, sP);
    near_work<S, Q, kForce>(sP, sp, red, s_links, ls, s_next);
    advance_step_when_last(B.ctr + 2, B.ctr);
}

// plain_chunk consecutive spans of the concatenated span ranges of all cases
// per CTA.  A span is BRICK consecutive node indices of one case, so each
// warp's loads and stores cover whole 128-byte rows whatever the box's nx
// (bricks of a box whose nx is not a multiple of 32 leave lanes idle and
// start rows mid-line); a node the near sweep takes (its brick is in the
// skip set) is left out.  The plain path needs only a few of a case's
// parameters, so they are read straight from the table (L1-cached) instead of
// copied to shared memory; the span's case comes from a per-span map.  The
// last CTA advances the plain sweep's step counter.
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 4) k_sweep_plain_batch(BatchArgs B) {
    const int total = B.span_off[B.ncases];
    const unsigned step = *(volatile const unsigned *)(B.ctr + 1);
    const Params *row = B.tab + (size_t)(step & 1) * B.ncases;
    const int g0 = blockIdx.x * B.plain_chunk;
    const int g1 = min(total, g0 + B.plain_chunk);
    // the case's parameters in shared memory (re-read when the CTA's spans
    // cross into the next case): loads from there cannot alias the stores to
    // the populations, so they stay in registers
    __shared__ Params sP;
    int cur = -1;
    for (int g = g0; g < g1; g++) {
        const int c = B.span_case[g];
        if (c != cur) {
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(row + c);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int k = threadIdx.x; k < (int)(sizeof(Params) / 4); k += blockDim.x) dst[k] = src[k];
            __syncthreads();
            cur = c;
        }
        const Params &P = sP;
        const int n = (g - B.span_off[c]) * BRICK + (int)threadIdx.x;
        if (n >= P.N) continue;
        const int nxy = P.nx * P.ny;
        const int z = n / nxy, r = n - z * nxy;
        const int y = r / P.nx, x = r - y * P.nx;
        const int b = x / BX + P.nbx * (y / BY + P.nby * (z / BZ));
        if (P.plain_spec) {  // pulls issued with the skip entry (see plain_brick)
            const bool skipped = P.skip[(step % 3) * P.nbricks + b] == (int)step;
            typename Codec<S>::C fin[Q];
            plain_pull<S, Q, true>(P, x, y, z, n, fin);
            if (!skipped) collide_store<S, Q, kForce, true>(P, fin, (S *)P.fB, P.N, n);
            continue;
        }
        if (P.skip[(step % 3) * P.nbricks + b] == (int)step) continue;  // the near sweep takes it
        plain_node<S, Q, kForce, true>(P, x, y, z, n);
    }
    advance_step_when_last(B.ctr + 3, B.ctr + 1);
}

}  // namespace lbmmb
