// hj_kernels.cuh -- kernels of one solve: the fused stage pass (K2), the
// alpha reductions (K1) and their launch helpers.  Instantiated per model in
// kern_<model>.cu so that the translation units compile in parallel.
#pragma once

#include "hj_device.cuh"
#include "odp_launch.h"

namespace odp {

// Fused stage pass (Algorithm 1, one Euler or TVD-RK2 stage, Section 3.1.3):
// derivatives, pbar, H, Lax-Friedrichs dissipation with the grid alpha,
// update and, on the last stage of a step of a tube, the min with l.
//   stage 0: Euler        phi' = phi + dt L(phi)              (cur -> nxt)
//   stage 1: RK2 stage 1  phi1 = phi + dt L(phi)              (cur -> nxt)
//   stage 2: RK2 stage 2  phi' = (phi + phi1 + dt L(phi1))/2  (nxt, cur -> cur)
template <int ND, int ORDER, int DYN>
__global__ void __launch_bounds__(256) k_stage(GridDesc g, DynDesc dy, SolveState *st,
                                               const float *__restrict__ l, int stage, int brt)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= uint32_t(g.total)) return;
    const float *__restrict__ src = (stage == 2) ? st->nxt : st->cur;
    float *dst = (stage == 2) ? st->cur : st->nxt;
    const unsigned *ab = st->alpha_bits[stage == 2 ? 1 : 0];

    int idx[ND];
    unflatten(g, ND, i, idx);
    float pm[ND], pp[ND], pbar[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        one_sided<ORDER>(src, int(i), idx[d], g.stride[d], g.n[d], g.periodic[d], g.inv_dz[d],
                         pm[d], pp[d]);
        pbar[d] = 0.5f * (pp[d] + pm[d]);
    }
    const float h = hamiltonian<DYN, ND>(g, dy, idx, pbar);
    float diss = 0.0f;
#pragma unroll
    for (int d = 0; d < ND; ++d) diss += __uint_as_float(ab[d]) * (pp[d] - pm[d]);
    const float L = h + 0.5f * diss;
    const float dt = float(st->dt);
    float v = src[i] + dt * L;
    if (stage == 2) v = 0.5f * (st->cur[i] + v);
    if (!isfinite(v)) atomicOr(&st->flags, FLAG_NONFINITE);
    if (brt && stage != 1) v = fminf(v, __ldg(l + i));
    dst[i] = v;
}

// Grid-wide max of the static alpha components into both stage slots.
template <int ND, int DYN>
__global__ void __launch_bounds__(256) k_alpha_static(GridDesc g, DynDesc dy, SolveState *st)
{
    __shared__ float red[8][ND];
    float a[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) a[d] = 0.0f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < uint32_t(g.total);
         i += gridDim.x * blockDim.x) {
        int idx[ND];
        unflatten(g, ND, i, idx);
        float la[ND];
        static_alpha<DYN, ND>(g, dy, idx, la);
#pragma unroll
        for (int d = 0; d < ND; ++d) a[d] = fmaxf(a[d], la[d]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        a[d] = warp_max(a[d]);
        if (lane == 0) red[warp][d] = a[d];
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        float m = 0.0f;
        for (int w = 0; w < (blockDim.x >> 5); ++w) m = fmaxf(m, red[w][threadIdx.x]);
        atomicMax(&st->alpha_bits[0][threadIdx.x], __float_as_uint(m));
        atomicMax(&st->alpha_bits[1][threadIdx.x], __float_as_uint(m));
    }
}

// Rel6D heading-rate alpha of phi (slot 0: cur, slot 1: nxt = phi1).
template <int ORDER>
__global__ void __launch_bounds__(256) k_alpha_rel6d(GridDesc g, DynDesc dy, SolveState *st, int slot)
{
    __shared__ float red[8];
    const float *__restrict__ src = slot ? st->nxt : st->cur;
    float a = 0.0f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < uint32_t(g.total);
         i += gridDim.x * blockDim.x) {
        int idx[6];
        unflatten(g, 6, i, idx);
        float pm, pp;
        one_sided<ORDER>(src, int(i), idx[2], g.stride[2], g.n[2], g.periodic[2], g.inv_dz[2], pm, pp);
        const float wp = __ldg(g.coord[4] + idx[4]);
        a = fmaxf(a, rel6d_theta_alpha(dy, wp, fminf(pm, pp), fmaxf(pm, pp)));
    }
    a = warp_max(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int w = 0; w < (blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        atomicMax(&st->alpha_bits[slot][2], __float_as_uint(m));
    }
}

inline int blocks_for(int64_t n, int threads) { return int((n + threads - 1) / threads); }

inline int reduce_blocks(int64_t n)
{
    const int b = blocks_for(n, 256);
    return b < 152 * 8 ? b : 152 * 8;
}

template <int ND, int DYN>
cudaError_t launch_stage_t(const GridDesc &g, const DynDesc &dy, SolveState *st, const float *l,
                           int order, int stage, int brt, cudaStream_t s)
{
    const int blocks = blocks_for(g.total, 256);
    if (order == 1)
        k_stage<ND, 1, DYN><<<blocks, 256, 0, s>>>(g, dy, st, l, stage, brt);
    else
        k_stage<ND, 2, DYN><<<blocks, 256, 0, s>>>(g, dy, st, l, stage, brt);
    return cudaGetLastError();
}

template <int ND, int DYN>
cudaError_t launch_alpha_static_t(const GridDesc &g, const DynDesc &dy, SolveState *st, cudaStream_t s)
{
    k_alpha_static<ND, DYN><<<reduce_blocks(g.total), 256, 0, s>>>(g, dy, st);
    return cudaGetLastError();
}

}  // namespace odp
