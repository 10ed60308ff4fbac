// Host check of the stage kernels' shared-window derivative helpers: the
// last-axis routine (axis_last, four nodes from one eight-node window, node
// pairs in paired arithmetic), the paired routine (pair_diffs) and the
// four-node routine fed with precomputed differences (segment_axis_d, the
// bulk-staged pass's stream axis) must give, bit for bit, what the one-node
// definition (diffs) and the five-row routine (segment_axis) give, followed
// by the Lax-Friedrichs terms of the axis.  Runs on the CPU: the
// helpers are __host__ __device__ and every paired operation is, lane by
// lane, the scalar IEEE operation.  Exit status 0 when all cases agree.
#include <cstdio>
#include <cstring>
#include <random>

#include "hj_kernels.cuh"

using namespace odp;

static float term(float dm, float dp, float cA, float cS, float cD, float L, bool has_a, bool has_s)
{
    const float P = dp + dm, M = dp - dm;
    float acc = L;
    if (has_a) acc = fmaf(cA, P, acc);
    if (has_s) acc = fmaf(cS, fabsf(P), acc);
    return fmaf(cD, M, acc);
}

template <int O>
static long check(std::mt19937 &rng, int cases)
{
    std::uniform_real_distribution<float> u(-1.0f, 1.0f);
    long bad = 0;
    for (int it = 0; it < cases; ++it) {
        // every third case on a coarse lattice, so that equal-magnitude
        // second differences (the ENO2 tie) occur often
        const bool coarse = it % 3 == 0;
        float w[8], cA[4], cDn[4], L[4], Lref[4];
        for (int j = 0; j < 8; ++j) w[j] = coarse ? float(int(u(rng) * 4.0f)) * 0.25f : u(rng);
        for (int k = 0; k < 4; ++k) {
            cA[k] = u(rng);
            cDn[k] = u(rng);
            L[k] = Lref[k] = u(rng);
        }
        const float cS = u(rng), cD = u(rng);
        const bool has_a = it & 1, has_s = (it >> 1) & 1, per_node = (it >> 2) & 1;
        float P[4];
        axis_last<O>(w, cA, cS, cD, L, has_a, has_s, P, per_node ? cDn : nullptr);
        for (int k = 0; k < 4; ++k) {
            float dm, dp;
            diffs<O>(w[k], w[k + 1], w[k + 2], w[k + 3], w[k + 4], dm, dp);
            const float r = term(dm, dp, cA[k], cS, per_node ? cDn[k] : cD, Lref[k], has_a, has_s);
            const float pr = dp + dm;
            if (memcmp(&r, &L[k], 4) != 0 || memcmp(&pr, &P[k], 4) != 0) ++bad;
        }
        // two windows at once through the paired routine
        float2 dm2, dp2;
        pair_diffs<O>(make_float2(w[0], w[3]), make_float2(w[1], w[4]), make_float2(w[2], w[5]),
                      make_float2(w[3], w[6]), make_float2(w[4], w[7]), dm2, dp2);
        float dma, dpa, dmb, dpb;
        diffs<O>(w[0], w[1], w[2], w[3], w[4], dma, dpa);
        diffs<O>(w[3], w[4], w[5], w[6], w[7], dmb, dpb);
        if (memcmp(&dma, &dm2.x, 4) || memcmp(&dpa, &dp2.x, 4) || memcmp(&dmb, &dm2.y, 4) ||
            memcmp(&dpb, &dp2.y, 4))
            ++bad;
        // four nodes from five rows, and from the differences of those rows
        // taken with the operations the callers of segment_axis_d use
        float4 r[5];
        for (int q = 0; q < 5; ++q)
            r[q] = make_float4(w[q], w[(q + 1) & 7], w[(q + 2) & 7], w[(q + 3) & 7]);
        auto sub = [](const float4 &x, const float4 &y) {
            return make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
        };
        const float4 a4 = sub(r[2], r[1]), b4 = sub(r[3], r[2]);
        const float4 d2l = sub(a4, sub(r[1], r[0])), d2m = sub(b4, a4), d2r = sub(sub(r[4], r[3]), b4);
        float2 A01 = make_float2(Lref[0], Lref[1]), A23 = make_float2(Lref[2], Lref[3]);
        float2 B01 = A01, B23 = A23;
        segment_axis<O>(r[0], r[1], r[2], r[3], r[4], cA, cS, cD, A01, A23, has_a, has_s);
        segment_axis_d<O>(a4, b4, d2l, d2m, d2r, cA, cS, cD, B01, B23, has_a, has_s);
        if (memcmp(&A01, &B01, 8) || memcmp(&A23, &B23, 8)) ++bad;
    }
    return bad;
}

int main()
{
    std::mt19937 rng(20220412u);
    const long b1 = check<1>(rng, 100000), b2 = check<2>(rng, 100000);
    printf("mismatches: upwind %ld, ENO2 %ld\n", b1, b2);
    return (b1 || b2) ? 1 : 0;
}
