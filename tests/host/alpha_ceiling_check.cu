// Host check of the premise behind the early exit of the Rel6D heading-rate
// alpha pass: the grid maximum of the per-node bound (rel6d_theta_alpha, the
// kernels' own function, on the float node coordinates of the w_p axis)
// never exceeds the ceiling the library computes once per dynamics
// (rel6d_heading_ceiling), and a node whose one-sided differences straddle
// zero reaches it exactly.  Then a CTA that finds the running maximum at the
// ceiling may skip its reads without changing the result.  Seeded grids and
// derivative intervals; exit status 0 when every case holds.
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "hj_device.cuh"
#include "odp_internal.h"

using namespace odp;

int main()
{
    std::mt19937 rng(11u);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    long fails = 0, cases = 0;
    for (int it = 0; it < 3000; ++it) {
        const int periodic = it % 5 == 0;
        const int n = periodic ? 1 + int(u(rng) * 60) : 2 + int(u(rng) * 60);
        const double lo = -3.0 * u(rng), hi = lo + 0.1 + 6.0 * u(rng);
        DynDesc dy{};
        dy.kind = DYN_REL6D;
        dy.dmode = (it & 1) ? MODE_MAX : MODE_MIN;
        dy.prm[3] = float(3.0 * u(rng));
        const float cap = rel6d_heading_ceiling(dy.prm[3], lo, hi, n, periodic);
        // the float node coordinates as the grid's table holds them
        const double h = periodic ? (hi - lo) / double(n) : (hi - lo) / double(n - 1);
        std::vector<float> wp(n);
        for (int i = 0; i < n; ++i) wp[i] = float(lo + double(i) * h);
        float reached = 0.0f;
        for (int i = 0; i < n; ++i) {
            reached = fmaxf(reached, rel6d_theta_alpha(dy, wp[i], -1.0f, 1.0f));   // straddling
            for (int k = 0; k < 8; ++k) {
                float a = float(4.0 * u(rng) - 2.0), b = float(4.0 * u(rng) - 2.0);
                if (k == 0) a = b = 0.0f;
                if (k == 1) a = 0.0f;
                if (a > b) std::swap(a, b);
                const float v = rel6d_theta_alpha(dy, wp[i], a, b);
                ++cases;
                if (!(v <= cap)) {
                    if (fails < 10) printf("bound %g above the ceiling %g (w_p %g)\n", v, cap, wp[i]);
                    ++fails;
                }
            }
        }
        if (memcmp(&reached, &cap, sizeof cap) != 0) {
            if (fails < 10) printf("the straddling maximum %g differs from the ceiling %g\n", reached, cap);
            ++fails;
        }
    }
    printf("cases %ld, failures %ld\n", cases, fails);
    return fails ? 1 : 0;
}
