// Launch wrappers of the storage-templated kernels; each sweep_<type>.cu
// instantiates them for one storage type.
#pragma once

#include "k_batch.cuh"
#include "k_static.cuh"

namespace lbmmb {

// SMs of the current device, queried once per device (152 on GB300; the
// value is only a grid-size choice, so a failed query falls back to it).
inline int sm_count() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cache[dev] = n;
    }
    return cache[dev];
}
// grid of the grid-stride kernels: eight CTAs per SM
inline int grid_stride_blocks() { return sm_count() * 8; }

template <typename S>
void launch_init_t(const Params &P, void *f, cudaStream_t st) {
    if (P.Q == 19) k_init<S, 19><<<grid_stride_blocks(), 256, 0, st>>>(P, (S *)f);
    else k_init<S, 15><<<grid_stride_blocks(), 256, 0, st>>>(P, (S *)f);
}
template <typename S>
void launch_flags_t(const Params &P, cudaStream_t st) {
    const int cap = P.chain_grid > 0 ? P.chain_grid : grid_stride_blocks() / 2;
    const int grid = P.nbricks < cap ? P.nbricks : cap;
    if (P.Q == 19) k_flags<S, 19><<<grid, BRICK, 0, st>>>(P);
    else k_flags<S, 15><<<grid, BRICK, 0, st>>>(P);
}
template <typename S>
void launch_sweep_plain_t(const Params &P, cudaStream_t st) {
    const bool force = P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0;
    const int grid = P.plain_grid > 0 && P.plain_grid < P.nbricks ? P.plain_grid : P.nbricks;
    if (P.Q == 19) {
        if (force) k_sweep_plain<S, 19, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_plain<S, 19, false><<<grid, BRICK, 0, st>>>(P);
    } else {
        if (force) k_sweep_plain<S, 15, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_plain<S, 15, false><<<grid, BRICK, 0, st>>>(P);
    }
}
template <typename S>
void launch_sweep_near_t(const Params &P, cudaStream_t st) {
    const bool force = P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0;
    const int cap = P.chain_grid > 0 ? P.chain_grid : kNearCtasPerSm * sm_count();
    const int grid = P.nbricks < cap ? P.nbricks : cap;
    if (P.Q == 19) {
        if (force) k_sweep_near<S, 19, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_near<S, 19, false><<<grid, BRICK, 0, st>>>(P);
    } else {
        if (force) k_sweep_near<S, 15, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_near<S, 15, false><<<grid, BRICK, 0, st>>>(P);
    }
}
// persistent, at the plain sweep's occupancy (4 CTAs per SM)
template <typename S>
void launch_sweep_near_plain_t(const Params &P, cudaStream_t st) {
    const bool force = P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0;
    const int cap = 4 * sm_count();
    const int grid = P.nbricks < cap ? P.nbricks : cap;
    if (P.Q == 19) {
        if (force) k_sweep_near_plain<S, 19, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_near_plain<S, 19, false><<<grid, BRICK, 0, st>>>(P);
    } else {
        if (force) k_sweep_near_plain<S, 15, true><<<grid, BRICK, 0, st>>>(P);
        else k_sweep_near_plain<S, 15, false><<<grid, BRICK, 0, st>>>(P);
    }
}
template <typename S>
void launch_fields_t(const Params &P, const void *f, const uint16_t *flags, double *rho, double *u, uint16_t *fl,
                     cudaStream_t st) {
    if (P.Q == 19) k_fields<S, 19><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, flags, rho, u, fl);
    else k_fields<S, 15><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, flags, rho, u, fl);
}
template <typename S>
void launch_get_pop_t(const Params &P, const void *f, double *out, cudaStream_t st) {
    if (P.Q == 19) k_get_pop<S, 19><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, out);
    else k_get_pop<S, 15><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, out);
}
template <typename S>
void launch_set_pop_t(const Params &P, void *f, const double *in, cudaStream_t st) {
    if (P.Q == 19) k_set_pop<S, 19><<<grid_stride_blocks(), 256, 0, st>>>(P, (S *)f, in);
    else k_set_pop<S, 15><<<grid_stride_blocks(), 256, 0, st>>>(P, (S *)f, in);
}
template <typename S>
void launch_check_t(const Params &P, const void *f, const uint16_t *flags, cudaStream_t st) {
    if (P.Q == 19) k_check<S, 19><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, flags);
    else k_check<S, 15><<<grid_stride_blocks(), 256, 0, st>>>(P, (const S *)f, flags);
}

template <typename S>
void launch_flags_batch_t(const BatchArgs &B, int Q, cudaStream_t st) {
    const int grid = B.ncases * B.g_chain;
    if (Q == 19) k_flags_batch<S, 19><<<grid, BRICK, 0, st>>>(B);
    else k_flags_batch<S, 15><<<grid, BRICK, 0, st>>>(B);
}
template <typename S>
void launch_near_batch_t(const BatchArgs &B, int Q, bool force, cudaStream_t st) {
    const int grid = B.ncases * B.g_chain;
    if (Q == 19) {
        if (force) k_sweep_near_batch<S, 19, true><<<grid, BRICK, 0, st>>>(B);
        else k_sweep_near_batch<S, 19, false><<<grid, BRICK, 0, st>>>(B);
    } else {
        if (force) k_sweep_near_batch<S, 15, true><<<grid, BRICK, 0, st>>>(B);
        else k_sweep_near_batch<S, 15, false><<<grid, BRICK, 0, st>>>(B);
    }
}
template <typename S>
void launch_plain_batch_t(const BatchArgs &B, int Q, bool force, int grid, cudaStream_t st) {
    if (Q == 19) {
        if (force) k_sweep_plain_batch<S, 19, true><<<grid, BRICK, 0, st>>>(B);
        else k_sweep_plain_batch<S, 19, false><<<grid, BRICK, 0, st>>>(B);
    } else {
        if (force) k_sweep_plain_batch<S, 15, true><<<grid, BRICK, 0, st>>>(B);
        else k_sweep_plain_batch<S, 15, false><<<grid, BRICK, 0, st>>>(B);
    }
}

template <typename S>
void launch_static_build_t(const Params &P, cudaStream_t st) {
    const int cap = grid_stride_blocks() / 2;
    const int grid = P.nbricks < cap ? P.nbricks : cap;
    if (P.Q == 19) k_static_build<S, 19><<<grid, BRICK, 0, st>>>(P);
    else k_static_build<S, 15><<<grid, BRICK, 0, st>>>(P);
}
template <typename S>
void launch_static_plain_t(const Params &P, cudaStream_t st) {
    const bool force = P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0;
    const int grid = (int)((P.N + BRICK - 1) / BRICK);
    if (P.Q == 19) {
        if (force) k_static_plain<S, 19, true><<<grid, BRICK, 0, st>>>(P);
        else k_static_plain<S, 19, false><<<grid, BRICK, 0, st>>>(P);
    } else {
        if (force) k_static_plain<S, 15, true><<<grid, BRICK, 0, st>>>(P);
        else k_static_plain<S, 15, false><<<grid, BRICK, 0, st>>>(P);
    }
}
template <typename S>
void launch_static_links_t(const Params &P, cudaStream_t st) {
    const bool force = P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0;
    const int warps = (P.snodes_n + kStaticNodesPerWarp - 1) / kStaticNodesPerWarp;
    const int cap = kNearCtasPerSm * sm_count();
    int grid = (warps + BRICK / 32 - 1) / (BRICK / 32);
    grid = grid < 1 ? 1 : (grid > cap ? cap : grid);
    if (P.Q == 19) {
        if (force) k_static_links<S, 19, true><<<grid, BRICK, 0, st>>>(P);
        else k_static_links<S, 19, false><<<grid, BRICK, 0, st>>>(P);
    } else {
        if (force) k_static_links<S, 15, true><<<grid, BRICK, 0, st>>>(P);
        else k_static_links<S, 15, false><<<grid, BRICK, 0, st>>>(P);
    }
}

template <typename S>
void launch_static_plain_batch_t(const BatchArgs &B, int Q, bool force, int grid, cudaStream_t st) {
    if (Q == 19) {
        if (force) k_static_plain_batch<S, 19, true><<<grid, BRICK, 0, st>>>(B);
        else k_static_plain_batch<S, 19, false><<<grid, BRICK, 0, st>>>(B);
    } else {
        if (force) k_static_plain_batch<S, 15, true><<<grid, BRICK, 0, st>>>(B);
        else k_static_plain_batch<S, 15, false><<<grid, BRICK, 0, st>>>(B);
    }
}
template <typename S>
void launch_static_links_batch_t(const BatchArgs &B, int Q, bool force, int warps, cudaStream_t st) {
    const int grid = (warps + BRICK / 32 - 1) / (BRICK / 32);
    if (Q == 19) {
        if (force) k_static_links_batch<S, 19, true><<<grid, BRICK, 0, st>>>(B);
        else k_static_links_batch<S, 19, false><<<grid, BRICK, 0, st>>>(B);
    } else {
        if (force) k_static_links_batch<S, 15, true><<<grid, BRICK, 0, st>>>(B);
        else k_static_links_batch<S, 15, false><<<grid, BRICK, 0, st>>>(B);
    }
}

#define LBMMB_INSTANTIATE(S)                                                                                     \
    template void launch_init_t<S>(const Params &, void *, cudaStream_t);                                        \
    template void launch_flags_t<S>(const Params &, cudaStream_t);                                               \
    template void launch_sweep_plain_t<S>(const Params &, cudaStream_t);                                         \
    template void launch_sweep_near_t<S>(const Params &, cudaStream_t);                                          \
    template void launch_sweep_near_plain_t<S>(const Params &, cudaStream_t);                                    \
    template void launch_fields_t<S>(const Params &, const void *, const uint16_t *, double *, double *,         \
                                     uint16_t *, cudaStream_t);                                                  \
    template void launch_get_pop_t<S>(const Params &, const void *, double *, cudaStream_t);                     \
    template void launch_set_pop_t<S>(const Params &, void *, const double *, cudaStream_t);                     \
    template void launch_check_t<S>(const Params &, const void *, const uint16_t *, cudaStream_t);             \
    template void launch_flags_batch_t<S>(const BatchArgs &, int, cudaStream_t);                                  \
    template void launch_near_batch_t<S>(const BatchArgs &, int, bool, cudaStream_t);                             \
    template void launch_plain_batch_t<S>(const BatchArgs &, int, bool, int, cudaStream_t);                       \
    template void launch_static_build_t<S>(const Params &, cudaStream_t);                                        \
    template void launch_static_plain_t<S>(const Params &, cudaStream_t);                                        \
    template void launch_static_links_t<S>(const Params &, cudaStream_t);                                        \
    template void launch_static_plain_batch_t<S>(const BatchArgs &, int, bool, int, cudaStream_t);               \
    template void launch_static_links_batch_t<S>(const BatchArgs &, int, bool, int, cudaStream_t);

}  // namespace lbmmb
