// Host check of the launch geometry of the single-solve stage passes: the
// plane-streaming pass (plane_geometry) and the bulk-staged pass
// (bulk_geometry, bulk_chunking) cut a grid into bands of rows, stream-axis
// chunks and outer-pencil blocks, and the kernels assume that these cover
// the grid exactly once.  For many seeded grid shapes this checks, with the
// library's own host functions: bands cover the rows with no empty band (and
// at least four rows a band in the plane pass), chunks cover the stream axis
// with no empty chunk and at least two planes in the last one (the window
// fill reads two ahead), at least four planes a chunk where the axis allows,
// CTA counts equal bands x chunks x pencils, the compute threads of a bulk
// CTA cover its band, pencil blocks tile every outer axis, and each fast
// division table divides like '/'; and the chunk counts the makespan model
// picks on the measured workloads.  Exit status 0 when every shape passes.
#include <cstdio>
#include <random>

#include "odp_internal.h"

using namespace odp;

static long fails = 0;
#define CHECK(c)                                                                      \
    do {                                                                              \
        if (!(c)) {                                                                   \
            if (fails < 20) printf("failed: %s (line %d, shape %s)\n", #c, __LINE__, shape); \
            ++fails;                                                                  \
        }                                                                             \
    } while (0)

static bool divides_like_slash(const FastDiv &f, uint32_t lim, std::mt19937 &rng)
{
    std::uniform_int_distribution<uint32_t> u(0, lim);
    for (int i = 0; i < 64; ++i) {
        const uint32_t x = i < 32 ? uint32_t(i) * f.d + uint32_t(i % 3) : u(rng);
        if (fast_div(x, f) != x / f.d) return false;
    }
    return true;
}

int main()
{
    std::mt19937 rng(7u);
    int shapes = 0, bulk_shapes = 0;
    for (int it = 0; it < 4000; ++it) {
        const int nd = 3 + it % 4;
        GridDesc D{};
        D.ndim = nd;
        std::uniform_int_distribution<int> side(nd == 6 ? 2 : 3, nd == 6 ? 30 : (nd == 5 ? 40 : 120));
        for (int d = 0; d < nd; ++d) D.n[d] = side(rng);
        if (it % 2 == 0) D.n[nd - 1] = (D.n[nd - 1] + 3) / 4 * 4;   // the bulk pass wants a multiple of 4
        D.n_pad = (D.n[nd - 1] + 3) / 4 * 4;
        D.segs = D.n_pad / 4;
        D.nr = D.n[nd - 2];
        D.periodic[nd - 3] = 0;
        D.periodic[nd - 2] = 0;
        char shape[96];
        int off = snprintf(shape, sizeof shape, "%d-D", nd);
        for (int d = 0; d < nd; ++d) off += snprintf(shape + off, sizeof shape - off, " %d", D.n[d]);
        const int sms = (it % 3 == 0) ? 152 : (it % 3 == 1 ? 76 : 1);
        long long pencils = 1;
        for (int d = 0; d < nd - 3; ++d) pencils *= D.n[d];
        const int ns = D.n[nd - 3], nr = D.nr;

        plane_geometry(D, sms);
        const PlaneGeom &pg = D.pg;
        if (pg.use) {
            ++shapes;
            CHECK(pg.rb >= 1 && pg.rb <= nr);
            CHECK(pg.rb * pg.nbands >= nr && (pg.nbands - 1) * pg.rb < nr);
            CHECK(pg.nbands == 1 || nr - (pg.nbands - 1) * pg.rb >= 4);
            CHECK(pg.threads % 32 == 0 && pg.threads >= pg.rb * D.segs && pg.threads <= 512);
            CHECK(pg.chunk >= 1 && pg.chunk * pg.nchunks >= ns && (pg.nchunks - 1) * pg.chunk < ns);
            CHECK(pg.chunk >= (ns < 4 ? ns : 4));
            CHECK((long long)pg.items == pencils * pg.nbands * pg.nchunks);
            CHECK(divides_like_slash(pg.div_nchunks, 1u << 30, rng) && pg.div_nchunks.d == uint32_t(pg.nchunks));
            CHECK(divides_like_slash(pg.div_nbands, 1u << 30, rng) && pg.div_nbands.d == uint32_t(pg.nbands));
            long long vol = 1;
            for (int d = 0; d < 3; ++d) {
                const bool outer = d < nd - 3;
                CHECK(pg.bdim[d] >= 1 && (!outer || D.n[d] % pg.bdim[d] == 0));
                CHECK(!outer || pg.nblk[d] * pg.bdim[d] == D.n[d]);
                CHECK(outer || (pg.bdim[d] == 1 && pg.nblk[d] == 1));
                vol *= pg.bdim[d];
            }
            CHECK(vol == pg.bvol);
        }

        bulk_geometry(D, sms, (it % 5 == 0) ? 128 : 256);
        const BulkGeom &bk = D.bk;
        if (bk.use) {
            ++bulk_shapes;
            CHECK(D.n[nd - 1] % 4 == 0 && pg.use);
            CHECK(bk.rb >= 1 && bk.rb * bk.nbands >= nr && (bk.nbands - 1) * bk.rb < nr);
            CHECK(bk.cwarps * 32 >= bk.rb * D.segs && bk.cwarps + 1 <= 16);
            CHECK(divides_like_slash(bk.div_nbands, 1u << 30, rng) && bk.div_nbands.d == uint32_t(bk.nbands));
            for (int o = 1; o <= 2; ++o) {
                if (!bk.smem[o - 1]) continue;
                CHECK(bk.smem[o - 1] == bulk_smem_bytes(bk, D.n_pad, nd, o, 3) && bk.smem[o - 1] <= 200 * 1024);
                for (int per_sm = 1; per_sm <= 8; per_sm += 3) {
                    bulk_chunking(D, o, per_sm, sms);
                    const int c = bk.chunk[o - 1], nc = bk.nchunks[o - 1];
                    CHECK(c >= 1 && c * nc >= ns && (nc - 1) * c < ns);
                    CHECK(nc == 1 || ns - (nc - 1) * c >= 2);
                    CHECK(c >= 4);
                    CHECK((long long)bk.items[o - 1] == pencils * bk.nbands * nc);
                    CHECK(bk.div_nchunks[o - 1].d == uint32_t(nc) && divides_like_slash(bk.div_nchunks[o - 1], 1u << 30, rng));
                }
            }
        }
    }
    // the chunk counts the makespan model picks on the measured workloads:
    // DubinsCar4D 80x80x40x64 (ENO2) with bands of 256 threads and two CTAs
    // per SM -> 5 chunks, with bands of 128 threads and four CTAs -> 3;
    // Rel6D 24^6 (upwind) with three CTAs per SM -> 1
    {
        const char *shape = "measured workloads";
        GridDesc D{};
        D.ndim = 4;
        const int n4[4] = {80, 80, 40, 64};
        for (int d = 0; d < 4; ++d) D.n[d] = n4[d];
        D.n_pad = 64;
        D.segs = 16;
        D.nr = 40;
        plane_geometry(D, 152);
        bulk_geometry(D, 152, 256);
        CHECK(D.bk.use && D.bk.nbands == 3);
        bulk_chunking(D, 2, 2, 152);
        CHECK(D.bk.nchunks[1] == 5);
        bulk_geometry(D, 152, 128);
        CHECK(D.bk.use && D.bk.nbands == 5 && D.bk.cwarps == 4);
        bulk_chunking(D, 2, 4, 152);
        CHECK(D.bk.nchunks[1] == 3);
        GridDesc R{};
        R.ndim = 6;
        for (int d = 0; d < 6; ++d) R.n[d] = 24;
        R.periodic[2] = 1;
        R.n_pad = 24;
        R.segs = 6;
        R.nr = 24;
        plane_geometry(R, 152);
        bulk_geometry(R, 152, 256);
        CHECK(R.bk.use && R.bk.nbands == 1 && R.bk.cwarps == 5);
        bulk_chunking(R, 1, 3, 152);
        CHECK(R.bk.nchunks[0] == 1);
    }
    printf("shapes with a plane geometry: %d, with a bulk geometry: %d, failures: %ld\n", shapes, bulk_shapes,
           fails);
    return fails ? 1 : 0;
}
