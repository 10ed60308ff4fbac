// Host check of the stage kernels' shared-window derivative helpers: the
// last-axis routine (axis_last, four nodes from one eight-node window, node
// pairs in paired arithmetic) and the paired routine (pair_diffs) must give,
// bit for bit, what the one-node definition (diffs) gives at every node,
// followed by the Lax-Friedrichs terms of the axis.  Runs on the CPU: the
// helpers are __host__ __device__ and every paired operation is, lane by
// lane, the scalar IEEE operation.  Exit status 0 when all cases agree.
#include <cstdio>
#include <cstring>
#include <random>

#include "hj_device.cuh"

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
