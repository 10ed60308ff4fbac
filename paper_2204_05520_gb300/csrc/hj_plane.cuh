// hj_plane.cuh -- plane-streaming stage pass (K2) for grids of 3 or more
// dimensions whose last two axes ("the plane") fit in shared memory.
//
// A CTA owns one pencil: fixed indices of axes 0..nd-4, a chunk of axis nd-3
// (the stream axis).  It walks the chunk plane by plane.  The planes s-r ..
// s+r of the stream axis live in a shared-memory ring, each moved global ->
// shared by one bulk asynchronous copy (cp.async.bulk with an mbarrier
// counting the bytes) one step ahead of its use.  Ring planes outside a
// non-periodic axis are ghost planes formed in shared memory from the
// boundary and inner planes (Section 3.1.1); the output plane is copied into a
// halo-padded buffer whose halo rows and columns hold the wrap or ghost
// values of the two in-plane axes.  Neighbour planes along the remaining
// outer axes are read from global memory.
#pragma once

#include "hj_kernels.cuh"

namespace odp {

// ---------------------------------------------------------------------------
// bulk asynchronous copy and mbarrier (inline PTX, sm_90+ forms)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity, giving up after a bounded number
// of polls (the copies it waits for are then reported as failed).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 26); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ghost plane k cells outside boundary plane pb with inner plane pi (Section 3.1.1)
__device__ __forceinline__ void ghost_plane(float *dst, const float *pb, const float *pi, float k, int n,
                                            int tid, int nthreads)
{
    for (int i = tid; i < n; i += nthreads) dst[i] = keep_sign_ghost(pb[i], pi[i], k);
}

// Neighbour plane of an outer axis, read straight from global memory: the
// plane delta elements away, or the ghost plane k cells outside the boundary
// from the planes db (boundary) and di (inner) away (Section 3.1.1).
struct NbPlane {
    long long delta, db, di;
    float k;
    int ghost;
};

__device__ __forceinline__ float4 nb_value(const float *__restrict__ src, long long gi, const NbPlane &q)
{
    if (!q.ghost) return ldg4(src + gi + q.delta);
    const float4 pb = ldg4(src + gi + q.db), pi = ldg4(src + gi + q.di);
    return make_float4(keep_sign_ghost(pb.x, pi.x, q.k), keep_sign_ghost(pb.y, pi.y, q.k),
                       keep_sign_ghost(pb.z, pi.z, q.k), keep_sign_ghost(pb.w, pi.w, q.k));
}

// One plane-streaming stage pass.  ND >= 3.
//
// Shared memory holds the ring of stream-axis planes (2r+2 slots: the 2r+1 in
// use and the next one, prefetched by a bulk copy while the current plane is
// computed; two mbarriers alternate between consecutive planes) and the
// halo-padded copy of the output plane.  Neighbour planes of the other outer
// axes are used once per output plane, so they are read straight from global
// memory (16-byte loads through the read-only path).
template <int ND, int ORDER, int DYN>
__global__ void __launch_bounds__(256) k_stage_plane(GridDesc g, DynDesc dy, SolveState *st,
                                                     const float *__restrict__ l, int stage, int brt)
{
    const PlaneGeom &pg = g.pg;
    constexpr int O = ORDER;
    constexpr int RING = 2 * O + 2;
    constexpr int NOUT = ND - 3;            // outer axes read from global memory
    extern __shared__ __align__(16) float smem[];
    float *ring = smem;                                  // RING planes
    float *ctr = ring + RING * pg.plane;                 // (nr + 2 O) x cp, halo-padded output plane
    uint64_t *bar = reinterpret_cast<uint64_t *>(ctr + (g.nr + 2 * O) * pg.cp);   // two mbarriers

    const int tid = threadIdx.x, nth = blockDim.x;
    const float *__restrict__ src = (stage == 2) ? st->nxt : st->cur;
    float *dst = (stage == 2) ? st->cur : st->nxt;
    const float *prev = st->cur;
    const unsigned *ab = st->alpha_bits[stage == 2 ? 1 : 0];
    float cD[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) cD[d] = 0.5f * bits_to_float(ab[d]) * g.inv_dz[d];
    StageArgs A;
    A.src = src;
    A.prev = prev;
    A.dst = dst;
    A.l = l;
    A.dt = float(st->dt);
    A.stage = stage;
    A.brt = brt;

    // this CTA's pencil: outer indices of axes 0..ND-4 and its chunk of axis ND-3
    const uint32_t item = blockIdx.x;
    const uint32_t outer = fast_div(item, pg.div_nchunks);
    const int chunk = int(item - outer * uint32_t(pg.nchunks));
    int idx[ND];
    {
        uint32_t o = outer;
        for (int d = ND - 4; d > 0; --d) {
            const uint32_t q = fast_div(o, g.div[d]);
            idx[d] = int(o - q * uint32_t(g.n[d]));
            o = q;
        }
        if (ND >= 4) idx[0] = int(o);
    }
    const int sa = ND - 3;                    // stream axis
    const int s_begin = chunk * pg.chunk;
    const int s_end = min(pg.ns, s_begin + pg.chunk);
    const long long pencil = (long long)outer * pg.ns;   // plane index of (outer, s = 0)
    const uint32_t pbytes = uint32_t(pg.plane) * 4u;

    // neighbour planes of the outer axes (same for every plane of the chunk)
    NbPlane nbq[NOUT > 0 ? NOUT : 1][2 * O];
#pragma unroll
    for (int d = 0; d < NOUT; ++d) {
        int k = 0;
        for (int o = -O; o <= O; ++o) {
            if (o == 0) continue;
            NbPlane q{};
            int j = idx[d] + o;
            const long long sd = g.stride[d];
            if (g.periodic[d]) {
                while (j < 0) j += g.n[d];
                while (j >= g.n[d]) j -= g.n[d];
                q.delta = (long long)(j - idx[d]) * sd;
            } else if (j >= 0 && j < g.n[d]) {
                q.delta = (long long)(j - idx[d]) * sd;
            } else {
                const int b = j < 0 ? 0 : g.n[d] - 1, in = j < 0 ? 1 : g.n[d] - 2;
                q.ghost = 1;
                q.k = j < 0 ? float(-j) : float(j - (g.n[d] - 1));
                q.db = (long long)(b - idx[d]) * sd;
                q.di = (long long)(in - idx[d]) * sd;
            }
            nbq[d][k++] = q;
        }
    }

    auto ring_slot = [&](int p) -> float * {
        int q = p % RING;
        if (q < 0) q += RING;
        return ring + q * pg.plane;
    };
    auto plane_ptr = [&](int p) -> const float * { return src + (pencil + p) * (long long)pg.plane; };
    auto in_range = [&](int p, int *q) -> bool {
        int v = p;
        if (g.periodic[sa]) {
            while (v < 0) v += pg.ns;
            while (v >= pg.ns) v -= pg.ns;
        }
        *q = v;
        return v >= 0 && v < pg.ns;
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    uint32_t phase_bits = 0;   // bit b: parity of the next phase of bar[b]

    // the planes of the first output plane
    if (tid == 0) {
        fence_proxy_async();
        uint32_t bytes = 0;
        int q;
        for (int p = s_begin - O; p <= s_begin + O; ++p)
            if (in_range(p, &q)) bytes += pbytes;
        uint64_t *b0 = &bar[s_begin & 1];
        mbar_arrive_expect_tx(b0, bytes);
        for (int p = s_begin - O; p <= s_begin + O; ++p)
            if (in_range(p, &q)) bulk_g2s(ring_slot(p), plane_ptr(q), pbytes, b0);
    }

    bool ok = true;
    for (int s = s_begin; s < s_end && ok; ++s) {
        // prefetch the ring plane of the next output plane into the free slot
        if (tid == 0 && s + 1 < s_end) {
            fence_proxy_async();
            int q;
            const int p = s + 1 + O;
            uint64_t *b1 = &bar[(s + 1) & 1];
            const bool load = in_range(p, &q);
            mbar_arrive_expect_tx(b1, load ? pbytes : 0u);
            if (load) bulk_g2s(ring_slot(p), plane_ptr(q), pbytes, b1);
        }
        const int bsel = s & 1;
        const uint32_t par = (phase_bits >> bsel) & 1u;
        ok = __syncthreads_and(mbar_wait_bounded(&bar[bsel], par) ? 1 : 0) != 0;
        phase_bits ^= (1u << bsel);
        if (!ok) {
            if (tid == 0) atomicOr(&st->flags, FLAG_COPY);
            break;
        }

        // ghost planes of a non-periodic stream axis
        if (!g.periodic[sa]) {
            const int first = (s == s_begin) ? s - O : s + O;
            for (int p = first; p <= s + O; ++p) {
                if (p < 0) ghost_plane(ring_slot(p), ring_slot(0), ring_slot(1), float(-p), pg.plane, tid, nth);
                if (p >= pg.ns)
                    ghost_plane(ring_slot(p), ring_slot(pg.ns - 1), ring_slot(pg.ns - 2), float(p - pg.ns + 1),
                                pg.plane, tid, nth);
            }
            __syncthreads();
        }
        const float *center = ring_slot(s);

        // ---- halo-padded copy of the output plane -----------------------------
        const int nr = g.nr, npad = g.n_pad, nl = g.n[ND - 1], cp = pg.cp;
        float *c0 = ctr + O * cp + 4;          // row 0, column 0
        for (int u = tid; u < nr * (npad / 4); u += nth) {
            const int r = int(fast_div(uint32_t(u), g.div_segs));
            const int c = (u - r * (npad / 4)) * 4;
            *reinterpret_cast<float4 *>(c0 + r * cp + c) =
                *reinterpret_cast<const float4 *>(center + r * npad + c);
        }
        __syncthreads();
        // halo rows (axis ND-2) and halo columns (last axis)
        for (int u = tid; u < 2 * O * nl; u += nth) {
            const int h = u / nl, c = u - h * nl;                // h: 0..2O-1
            const int jr = (h < O) ? h - O : nr + (h - O);       // row outside [0, nr)
            float v;
            if (g.periodic[ND - 2]) {
                const int q = ((jr % nr) + nr) % nr;
                v = c0[q * cp + c];
            } else if (jr < 0) {
                v = keep_sign_ghost(c0[c], c0[cp + c], float(-jr));
            } else {
                v = keep_sign_ghost(c0[(nr - 1) * cp + c], c0[(nr - 2) * cp + c], float(jr - nr + 1));
            }
            c0[jr * cp + c] = v;
        }
        for (int u = tid; u < 2 * O * nr; u += nth) {
            const int r = u / (2 * O), h = u - r * (2 * O);
            const int jc = (h < O) ? h - O : nl + (h - O);
            float *rowp = c0 + r * cp;
            float v;
            if (g.periodic[ND - 1]) {
                const int q = ((jc % nl) + nl) % nl;
                v = rowp[q];
            } else if (jc < 0) {
                v = keep_sign_ghost(rowp[0], rowp[1], float(-jc));
            } else {
                v = keep_sign_ghost(rowp[nl - 1], rowp[nl - 2], float(jc - nl + 1));
            }
            rowp[jc] = v;
        }
        __syncthreads();

        // ---- per-node update --------------------------------------------------
        idx[sa] = s;
        const long long gplane = (pencil + s) * (long long)pg.plane;
        const float *rm1 = ring_slot(s - 1), *rp1 = ring_slot(s + 1);
        const float *rm2 = (O == 2) ? ring_slot(s - 2) : rm1, *rp2 = (O == 2) ? ring_slot(s + 2) : rp1;
        for (int u = tid; u < nr * (npad / 4); u += nth) {
            const int r = int(fast_div(uint32_t(u), g.div_segs));
            const int s0 = (u - r * (npad / 4)) * 4;
            idx[ND - 2] = r;
            idx[ND - 1] = s0;
            const int off = r * npad + s0;
            const long long gi = gplane + off;
            float cA[ND][4], cS[ND];
            drift<DYN, ND>(g, dy, idx, cA, cS);
            const float *C = c0 + r * cp + s0;
            const float4 c4 = *reinterpret_cast<const float4 *>(C);
            float2 L01 = make_float2(0.0f, 0.0f), L23 = make_float2(0.0f, 0.0f);

            // outer axes from global memory
#pragma unroll
            for (int d = 0; d < NOUT; ++d) {
                const float4 m1 = nb_value(src, gi, nbq[d][O - 1]);
                const float4 p1 = nb_value(src, gi, nbq[d][O]);
                const float4 m2 = (O == 2) ? nb_value(src, gi, nbq[d][0]) : m1;
                const float4 p2 = (O == 2) ? nb_value(src, gi, nbq[d][2 * O - 1]) : p1;
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[d], cS[d], cD[d], L01, L23, has_drift<DYN, ND>(d),
                                    has_bound<DYN, ND>(d));
            }
            // stream axis from the ring
            {
                const float4 m1 = *reinterpret_cast<const float4 *>(rm1 + off);
                const float4 p1 = *reinterpret_cast<const float4 *>(rp1 + off);
                const float4 m2 = (O == 2) ? *reinterpret_cast<const float4 *>(rm2 + off) : m1;
                const float4 p2 = (O == 2) ? *reinterpret_cast<const float4 *>(rp2 + off) : p1;
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[ND - 3], cS[ND - 3], cD[ND - 3], L01, L23,
                                    has_drift<DYN, ND>(ND - 3), has_bound<DYN, ND>(ND - 3));
            }
            // in-plane row axis (ND-2)
            {
                const float4 m1 = *reinterpret_cast<const float4 *>(C - cp);
                const float4 p1 = *reinterpret_cast<const float4 *>(C + cp);
                const float4 m2 = (O == 2) ? *reinterpret_cast<const float4 *>(C - 2 * cp) : m1;
                const float4 p2 = (O == 2) ? *reinterpret_cast<const float4 *>(C + 2 * cp) : p1;
                segment_axis<ORDER>(m2, m1, c4, p1, p2, cA[ND - 2], cS[ND - 2], cD[ND - 2], L01, L23,
                                    has_drift<DYN, ND>(ND - 2), has_bound<DYN, ND>(ND - 2));
            }
            // last axis: window w[j] = phi(s0 - 2 + j); halo columns are in place
            float L[4] = {L01.x, L01.y, L23.x, L23.y};
            {
                const float2 lh = *reinterpret_cast<const float2 *>(C - 2);
                const float2 rh = *reinterpret_cast<const float2 *>(C + 4);
                float w[8] = {lh.x, lh.y, c4.x, c4.y, c4.z, c4.w, rh.x, rh.y};
                // a partial last segment: the window continues with the halo columns
                if (s0 + 4 > nl) {
#pragma unroll
                    for (int j = 2; j < 8; ++j)
                        if (s0 + j - 2 >= nl) w[j] = C[j - 2];
                }
                axis_last<ORDER>(w, cA[ND - 1], cS[ND - 1], cD[ND - 1], L, has_drift<DYN, ND>(ND - 1),
                                 has_bound<DYN, ND>(ND - 1));
            }
            // update, Heun average, non-finite flag, BRT min
            const int nvalid = nl - s0 < 4 ? nl - s0 : 4;
            float4 out;
            if (stage_epilogue(A, int(gi), c4, L, nvalid, out)) atomicOr(&st->flags, FLAG_NONFINITE);
            if (nvalid == 4) {
                *reinterpret_cast<float4 *>(dst + gi) = out;
            } else {
                const float o[4] = {out.x, out.y, out.z, out.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < nvalid) dst[gi + k] = o[k];
            }
        }
        __syncthreads();
    }
}

}  // namespace odp
