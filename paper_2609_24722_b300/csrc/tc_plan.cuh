// tc_plan.cuh -- host planning of pair passes and device helpers shared by
// the libtc translation units.
#pragma once

#include <algorithm>
#include <vector>

#include "tc_internal.h"
#include "tc_pass.cuh"
#include "tc_pass_mixed.cuh"

namespace tc {

constexpr int kThreads = 256;       // pass CTA size = source tile length T
constexpr int kR = 2;               // rows per thread
constexpr int kRB = kThreads * kR;  // rows per row block
constexpr int kT = kThreads;

// ------------------------------------------------------------ planning ---

struct Plan {
    std::vector<Prob> prob;
    int64_t W = 0;   // total units
    int64_t G = 1;   // CTAs
    int64_t slots = 1;
    int64_t M = 0;   // total rows
};

// Fill unit offsets, row blocks and tile counts; W = sum of units.
inline void plan_units(Plan& P)
{
    int64_t u = 0;
    for (auto& p : P.prob) {
        p.n_rb = (int32_t)((p.m + kRB - 1) / kRB);
        p.n_t_snap = (int32_t)((p.snap_e - p.snap_b + kT - 1) / kT);
        p.n_t_priv = (int32_t)((p.m + kT - 1) / kT);
        p.unit_off = u;
        u += (int64_t)p.n_rb * (p.n_t_snap + p.n_t_priv);
    }
    P.W = u;
}

// Largest number of ranges that touch one row block, for G equal ranges over
// units [u_base, u_base + W) of problems `ps` (the slots a pass needs per row).
inline int64_t plan_slots(const std::vector<Prob>& ps, size_t first, size_t last, int64_t u_base, int64_t W,
                          int64_t G)
{
    int64_t best = 1;
    for (size_t s = first; s < last; ++s) {
        const Prob& p = ps[s];
        int64_t n_t = p.n_t_snap + p.n_t_priv;
        for (int64_t rb = 0; rb < p.n_rb; ++rb) {
            int64_t U0 = p.unit_off + rb * n_t - u_base;
            int64_t c = sk_owner(U0 + n_t - 1, W, G) - sk_owner(U0, W, G) + 1;
            best = std::max(best, c);
        }
    }
    return best;
}

// Ranges of a mixed pass whose persistent CTAs take them from a queue
// (PassArgs::ticket).  The count depends on the work and the SM count only, not
// on the launch shape, so every shape computes the same per-range sums; the
// queue keeps the SMs busy when units differ in cost (near tiles, partial row
// blocks).  It is k x 12 SMs ranges (k = 1 .. 5, ranges of at least
// kDynMinUnits units where the work allows), so that 3, 4, 5 or 6 resident
// CTAs per SM take them in whole rounds (mixed_ctas); below 12 SMs units, one
// range per unit.
constexpr int64_t kDynMinUnits = 16;
constexpr size_t kPassCtrOff = 96;  // the queue's ticket counter in the workspace counter area
inline int64_t mixed_ranges(int64_t W, int64_t min_units = kDynMinUnits, int64_t kmax = 5)
{
    const int64_t r0 = 12 * (int64_t)sm_count();
    if (W <= r0) return std::max<int64_t>(1, W);
    return std::min<int64_t>(kmax, std::max<int64_t>(1, W / (min_units * r0))) * r0;
}

// Ranges of the symmetric float64 pass: a unit there is ~1 ms of one CTA's
// float64 pipe and the units of the lower triangle cost nothing, so ranges of
// about 2 units (up to 20 x 12 SMs of them) keep the queue's tail short.
inline int64_t sym_ranges(int64_t W) { return mixed_ranges(W, 2, 20); }

// CTAs for `ranges` ranges when at most `ctas_max` are resident: as few rounds
// of the queue as ctas_max allows, with the ranges spread evenly over them.
inline int64_t mixed_ctas(int64_t ranges, int64_t ctas_max)
{
    const int64_t rounds = (ranges + ctas_max - 1) / ctas_max;
    return (ranges + rounds - 1) / rounds;
}

// ------------------------------------------------------- small kernels ---

__device__ __forceinline__ bool inside(double x, double y)
{
    double r = sqrt(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    return r <= 1.0 + kWallSlack;
}

// Deterministic block sum of one double per thread (fixed tree).
template <int THREADS> __device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// Number of slots holding partials of row block rb of problem p.
__device__ __forceinline__ int64_t slot_count(const Prob& p, int rb, int64_t u_base, int64_t W, int64_t G)
{
    int64_t n_t = p.n_t_snap + p.n_t_priv;
    int64_t U0 = p.unit_off + rb * n_t - u_base;
    return sk_owner(U0 + n_t - 1, W, G) - sk_owner(U0, W, G) + 1;
}

__device__ __forceinline__ double2 project1(double2 p, double radius, bool pinned)
{
    double r = sqrt(__dadd_rn(__dmul_rn(p.x, p.x), __dmul_rn(p.y, p.y)));
    if (pinned) {
        if (r > 0.0) return make_double2(p.x / r, p.y / r);
    } else if (r > radius) {
        double s = radius / r;
        return make_double2(__dmul_rn(p.x, s), __dmul_rn(p.y, s));
    }
    return p;
}

// Gradient with the wall-blocked components removed (pinned charges keep the
// component along the circle; a free charge at the wall whose force -g points
// outward keeps the tangential part).
__device__ __forceinline__ double2 wall_grad(double2 x, double2 g, double radius, bool pinned)
{
    double r = sqrt(__dadd_rn(__dmul_rn(x.x, x.x), __dmul_rn(x.y, x.y)));
    if (r > 0.0 && (pinned || r >= radius * (1.0 - 1e-12))) {
        double ux = x.x / r, uy = x.y / r;
        double gr = __dadd_rn(__dmul_rn(g.x, ux), __dmul_rn(g.y, uy));
        if (pinned || gr < 0.0) {
            g.x = __dsub_rn(g.x, __dmul_rn(gr, ux));
            g.y = __dsub_rn(g.y, __dmul_rn(gr, uy));
        }
    }
    return g;
}

// ------------------------------------------------------ pass launching ---

// Launch shapes of the float32 pass.  All keep the row block at kRB = 512
// rows and the tile at kT = 256 sources, so one plan serves every shape; they
// differ in threads per CTA and rows per thread (register blocking).
constexpr int kMixedConfigs = 6;
extern int g_mixed_config;  // chosen shape (tc_set_pass_config); 0 by default

template <bool WANT_E, bool WANT_G> struct MixedShape {
    using fn_t = void (*)(PassArgs, int64_t, int64_t);
    // (rows per thread, threads per CTA, minimum resident CTAs per SM)
    static fn_t kernel(int c, int* threads)
    {
        switch (c) {
            case 1: *threads = 256; return k_pass_mixed<2, 256, kT, 4, WANT_E, WANT_G>;
            case 2: *threads = 256; return k_pass_mixed<2, 256, kT, 6, WANT_E, WANT_G>;
            case 3: *threads = 128; return k_pass_mixed<4, 128, kT, 4, WANT_E, WANT_G>;
            case 4: *threads = 128; return k_pass_mixed<4, 128, kT, 6, WANT_E, WANT_G>;
            case 5: *threads = 64; return k_pass_mixed<8, 64, kT, 6, WANT_E, WANT_G>;
            default: *threads = 256; return k_pass_mixed<2, 256, kT, 3, WANT_E, WANT_G>;
        }
    }
};

// SYM: the float64 kernel with the symmetric (PassArgs::sym) path compiled in.
template <int KIND, bool WANT_E, bool WANT_G, bool SYM = false> inline auto pass_kernel(int* threads)
{
    if constexpr (KIND == PASS_MIXED) {
        return MixedShape<WANT_E, WANT_G>::kernel(g_mixed_config, threads);
    } else {
        *threads = kThreads;
        return k_pass<KIND, kR, kThreads, WANT_E, WANT_G, SYM && KIND == PASS_F64>;
    }
}

template <int KIND, bool WANT_E, bool WANT_G>
inline cudaError_t launch_pass(const PassArgs& a, int64_t G, int64_t u_base, int64_t row_sub, cudaStream_t s)
{
    if (a.W <= 0) return cudaSuccess;
    int threads = 0;
    auto fn = pass_kernel<KIND, WANT_E, WANT_G>(&threads);
    if (KIND == PASS_F64 && a.sym) fn = pass_kernel<KIND, WANT_E, WANT_G, true>(&threads);
    if (a.ticket) {
        PassArgs b = a;
        b.ranges = G;
        fn<<<(unsigned)std::min<int64_t>(a.ctas, G), threads, 0, s>>>(b, u_base, row_sub);
    } else {
        fn<<<(unsigned)G, threads, 0, s>>>(a, u_base, row_sub);
    }
    return cudaGetLastError();
}

template <int KIND, bool WANT_E, bool WANT_G, bool SYM = false> inline int64_t pass_grid(int64_t W)
{
    int threads = 0;
    auto fn = pass_kernel<KIND, WANT_E, WANT_G, SYM>(&threads);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    int64_t g = (int64_t)sm_count() * occ;
    return std::max<int64_t>(1, std::min<int64_t>(g, W));
}

}  // namespace tc
