// odp_common.cuh -- device-side data layout shared by the libodp kernels.
//
// A grid is a dense C-order float32 array (last axis fastest).  Kernels get a
// GridDesc by value (sizes, strides, reciprocal spacings, per-axis node
// tables) and a DynDesc (model id, input modes, parameters).  The mutable
// state of a solve (t, dt, step counters, alpha, ping-pong pointers, error
// flags) lives in one SolveState in device memory so that a captured CUDA
// graph can run the whole time loop without the host.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <cstring>

#define ODP_MAXD 6

// Per-node helpers are host+device so that the exact kernel arithmetic can
// also be stepped through on the host when debugging.
#define ODP_HD __host__ __device__ __forceinline__

namespace odp {

ODP_HD float ldgf(const float *p)
{
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

ODP_HD float4 ldg4(const float *p)
{
#ifdef __CUDA_ARCH__
    return __ldg(reinterpret_cast<const float4 *>(p));
#else
    return *reinterpret_cast<const float4 *>(p);
#endif
}

ODP_HD float2 ldg2(const float *p)
{
#ifdef __CUDA_ARCH__
    return __ldg(reinterpret_cast<const float2 *>(p));
#else
    return *reinterpret_cast<const float2 *>(p);
#endif
}

ODP_HD float bits_to_float(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, sizeof(f));
    return f;
#endif
}

enum DynKind { DYN_SINGLE_INT = 0, DYN_DUBINS3D = 1, DYN_DUBINSCAR4D = 2, DYN_REL6D = 3, DYN_ADVECTION = 4,
               DYN_CAPTURE = 5 };
enum Mode { MODE_MIN = 0, MODE_MAX = 1 };

// Error flags raised on the device.
enum : int { FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_COPY = 4 };

// Unsigned division by an invariant divisor through a multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l for
// every n < 2^31.
struct FastDiv {
    uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
}

ODP_HD uint32_t fast_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    const uint32_t hi = __umulhi(f.m, n);
#else
    const uint32_t hi = uint32_t((uint64_t(f.m) * uint64_t(n)) >> 32);
#endif
    return (hi + n) >> f.l;
}

// Geometry of the plane-streaming stage pass (hj_plane.cuh; host computed).
// A CTA covers a band of rb rows of the plane (the last band may be shorter,
// never below 4 rows) for a chunk of the stream axis at fixed outer indices.
struct PlaneGeom {
    int use;           // 1: the grid runs the plane-streaming pass
    int ns;            // length of the stream axis (axis ndim-3)
    int chunk;         // stream-axis planes per CTA
    int nchunks;       // ceil(ns / chunk)
    int rb;            // rows per band
    int nbands;        // ceil(nr / rb)
    int items;         // outer pencils * nbands * nchunks (CTAs per launch)
    int plane;         // floats per plane: nr * n_pad
    int cp;            // tile row pitch: n_pad + 4
    int threads;       // CTA size: rb * segs rounded up to a warp
    int smem[2];       // dynamic shared bytes (two tiles) for stencil radius 1, 2
    FastDiv div_nchunks, div_nbands;
    // outer pencils in blocks: bdim[d] indices of outer axis d per block,
    // nblk[d] blocks along it, bvol pencils per block
    int bdim[3], nblk[3], bvol;
    FastDiv div_bdim[3], div_nblk[3], div_bvol;
};

// Geometry of the bulk-staged stage pass of a single solve (hj_bulk.cuh;
// host computed).  Work items as in PlaneGeom (chunk fastest, then band,
// then outer pencil in C order); the CTA has cwarps compute warps and one
// producer warp; rc / rx ring slots hold centre and neighbour tiles.
struct BulkGeom {
    int use;           // 0: never; 1: where it is the faster pass (4 or more dims); 2: wherever it applies
    int rb, nbands;    // rows per band (the last band may be shorter), bands
    int chunk[2], nchunks[2];   // stream-axis chunking per stencil radius 1, 2
    int items[2];      // CTAs per launch, per stencil radius
    int cwarps;        // compute warps per CTA
    int rc, rx;        // ring slots
    int smem[2];       // dynamic shared bytes per stencil radius with all three read-once tiles (0: too large)
    FastDiv div_nchunks[2], div_nbands;
};

// Dynamic shared bytes of the bulk-staged pass: the barrier area, rc centre
// slots of rb + 2o rows, and rx neighbour slots of 2o (nd - 3) neighbour
// tiles and naux read-once tiles of rb rows each.
ODP_HD long long bulk_smem_bytes(const BulkGeom &bk, int n_pad, int nd, int o, int naux)
{
    const long long row = 4LL * n_pad;
    return 512 + bk.rc * (bk.rb + 2LL * o) * row + bk.rx * (2LL * o * (nd - 3) + naux) * bk.rb * row;
}

// Storage: C order with the last axis padded to n_pad, a multiple of 4 nodes,
// so that every row starts on a 16-byte boundary and a thread can move four
// consecutive nodes of a row with one vector access.  Padding lanes are never
// read as neighbours and never written by the stage kernels.
struct GridDesc {
    int ndim;
    int total;                   // number of nodes (< 2^31)
    int n_pad;                   // padded length of the last axis
    int rows;                    // product of n[0 .. ndim-2]
    int segs;                    // n_pad / 4: four-node segments per row
    int nthreads;                // rows * segs
    FastDiv div_segs;
    int n[ODP_MAXD];
    int stride[ODP_MAXD];        // C order over the padded storage: stride[ndim-1] == 1
    int periodic[ODP_MAXD];
    float inv_dz[ODP_MAXD];      // 1 / node spacing
    double dz[ODP_MAXD];         // node spacing (float64, for the CFL step)
    FastDiv div[ODP_MAXD];       // divisors n[d] for unflattening
    const float *coord[ODP_MAXD];  // node coordinates of each axis (device)
    const float *cos_tab;        // cos / sin of the angle axis nodes (device)
    const float *sin_tab;
    // per-node dissipation of the capture model: each node's coefficient
    // alpha_d / (2 h_d) per axis d, written by its alpha pass every stage
    // (3 arrays of cdn_stride floats at the nodes' storage offsets), or nullptr
    float *cdn;
    int cdn_stride;
    // geometry of the row-blocked stage pass: a thread owns one four-node
    // segment of the last axis in each of R consecutive rows of axis ndim-2
    // (a "row group"); threads are numbered segment fastest, then row group,
    // then plane (the remaining outer axes, product of n[0 .. ndim-3]).
    int R;
    int nr;                      // n[ndim-2] (1 for a 1-D grid)
    int row_groups;              // ceil(nr / R)
    int planes;
    int nthreads_rb;             // segs * row_groups * planes
    FastDiv div_row_groups;
    PlaneGeom pg;
    BulkGeom bk;
};

struct DynDesc {
    int kind;
    int umode, dmode;
    int angle_axis;              // axis holding the heading angle, -1 if none
    int local_diss;              // 1: per-node dissipation alpha_i (Algorithm 1's second loop)
    float prm[8];
    // the largest value the phi-dependent alpha component (Rel6D heading
    // rate) can take on this grid, in the kernels' float arithmetic; 0: none
    float acap;
};

// alpha is kept as the bit pattern of a non-negative float so that the
// grid-wide max is an atomicMax on unsigned integers.
struct SolveState {
    double t;                    // look-back time reached
    double t_end;                // end of the current tau segment
    double dt;                   // step of the current time step
    double cfl;
    long long steps;             // full steps taken over all segments
    long long max_steps;
    int seg;                     // current tau segment
    int n_seg;
    int last;                    // current step is the clipped last step of a segment
    int flags;                   // FLAG_* bits
    int snap_index;              // snapshot to write when the IF body runs
    int pad;
    float *cur;                  // phi^n
    float *nxt;                  // phi^{n+1} (Euler) or phi^1 (RK2)
    const double *tau;           // device copy of the tau schedule
    float *snapshots;            // n_tau * total floats, or nullptr
    unsigned alpha_bits[2][8];   // per stage slot (0: stage 1, 1: stage 2)
    unsigned alpha_last[8];      // alpha of the last stage of the last step
    int go;                      // the time loop continues (host-stepped loop)
    int snap_now;                // a snapshot is due after this step (host-stepped loop)
};

}  // namespace odp
