// tc_pass_mixed.cuh -- the mixed-precision pair pass (float32 pair terms).
//
// Same unit walk as k_pass (persistent CTAs, stream-K ranges, per-row-block
// partials), specialised for float32 arithmetic on the packed FP32x2 path of
// sm_100-class SMs (FADD2/FMUL2/FFMA2 via __fadd2_rn/__fmul2_rn/__ffma2_rn):
// each thread keeps its R rows as R/2 float2 pairs, and every source is
// staged in shared memory twice, as (-x_hi, -x_hi, -y_hi, -y_hi) and
// (-x_lo, -x_lo, -y_lo, -y_lo), so one LDS.128 yields both lanes of both
// coordinates.
//
// Near and far tiles.  A coordinate x is carried as x_hi + x_lo (float32 hi
// and lo parts).  The separation dx = x_i - x_j of two charges is formed as
// (x_hi,i - x_hi,j) + (x_lo,i - x_lo,j), accurate to a float32 rounding of dx
// itself.  For pairs at distance >= kFarDist the hi parts alone give dx to
// within 2^-24 absolute, a relative error below 3e-6 of the pair's term.  So a
// tile whose bounding box lies at least kFarDist from the row block's box
// skips the lo parts: 8 float32 lane operations and one MUFU.RSQ per ordered
// pair (dx, dy; r^2 as a mul and an fma; r^-3 as two muls; two gradient fmas),
// plus one add for the energy.  Near tiles (and the tiles holding the rows'
// own charges) add the lo parts and, where needed, drop the self pair.
#pragma once

#include "tc_device.cuh"

namespace tc {

constexpr float kFarDist = 0.02f;
constexpr float kBoxEmptyLo = 3.0e38f, kBoxEmptyHi = -3.0e38f;

// Packed rows of one thread: R rows as R/2 float2 pairs.  The pairs (hi and
// lo parts) and the cross-tile accumulators stay in shared memory
// (per-thread slots); each tile reads the pairs back with one LDS.64 each, so
// they occupy adjacent registers only while the tile loop runs.
template <int R> struct MixedRows {
    static_assert(R % 2 == 0, "rows come in pairs");
    static constexpr int P = R / 2;

    // Loads rows rl0 + r*rstride (r < R) when `holds`; rows past m, and every
    // row of a thread that holds none, sit far away.  The pairs go to
    // lo2[4P][stride] (x lo, y lo, x hi, y hi pairs), accumulators
    // acc[6R][stride] are zeroed.  Returns the box (xmin, ymin, xmax, ymax) of
    // the valid rows.
    __device__ float4 load(const float4* rows, int64_t base, int64_t rl0, int rstride, bool holds, int m,
                           float2* lo2, float* acc, int stride, int tid)
    {
        float4 box = make_float4(3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f);
        float4 q[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t rl = rl0 + (int64_t)r * rstride;
            const bool ok = holds && rl < m;
            q[r] = ok ? rows[base + rl] : make_float4(kFarRow32, kFarRow32, 0.f, 0.f);
            if (ok) {
                box.x = fminf(box.x, q[r].x);
                box.y = fminf(box.y, q[r].y);
                box.z = fmaxf(box.z, q[r].x);
                box.w = fmaxf(box.w, q[r].y);
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            lo2[p * stride + tid] = make_float2(q[2 * p].z, q[2 * p + 1].z);
            lo2[(P + p) * stride + tid] = make_float2(q[2 * p].w, q[2 * p + 1].w);
            lo2[(2 * P + p) * stride + tid] = make_float2(q[2 * p].x, q[2 * p + 1].x);
            lo2[(3 * P + p) * stride + tid] = make_float2(q[2 * p].y, q[2 * p + 1].y);
        }
#pragma unroll
        for (int c = 0; c < 6 * R; ++c) acc[c * stride + tid] = 0.f;
        return box;
    }

    // One tile of T sources.  hi[j] = (-x_hi, -x_hi, -y_hi, -y_hi), lo[j] the
    // same for the lo parts.  The tile sums (sum dx r^-3 = -grad, sum 1/r) are
    // folded into the shared accumulators acc[6R][stride] with TwoSum.  Row r
    // of the thread is source jself0 + r * rstride of a tile holding its own
    // charges (SELF).  Only the first PA pairs are computed: the caller passes
    // PA < P when every row of the later pairs lies past the end of the
    // problem (a partial last row block), so the CTA skips them together.
    template <int T, bool NEAR, bool SELF, bool WANT_E, bool WANT_G, int PA = P>
    __device__ __forceinline__ void tile(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                         const float2* lo2, float* acc, int stride, int tid, int jself0,
                                         int rstride, float escale)
    {
        static_assert(PA >= 1 && PA <= P, "active pairs");
        float2 et[PA], gxt[PA], gyt[PA], xl[PA], yl[PA], xh[PA], yh[PA];
#pragma unroll
        for (int p = 0; p < PA; ++p) {
            et[p] = gxt[p] = gyt[p] = make_float2(0.f, 0.f);
            xh[p] = lo2[(2 * P + p) * stride + tid];
            yh[p] = lo2[(3 * P + p) * stride + tid];
            if (NEAR) {
                xl[p] = lo2[p * stride + tid];
                yl[p] = lo2[(P + p) * stride + tid];
            }
        }
#pragma unroll 8
        for (int j = 0; j < T; ++j) {
            const float4 h = hi[j];
            const float2 qx = make_float2(h.x, h.y), qy = make_float2(h.z, h.w);
            float2 lx, ly;
            if (NEAR) {
                const float4 l = lo[j];
                lx = make_float2(l.x, l.y);
                ly = make_float2(l.z, l.w);
            }
#pragma unroll
            for (int p = 0; p < PA; ++p) {
                float2 dx = __fadd2_rn(xh[p], qx);
                float2 dy = __fadd2_rn(yh[p], qy);
                if (NEAR) {
                    dx = __fadd2_rn(dx, __fadd2_rn(xl[p], lx));
                    dy = __fadd2_rn(dy, __fadd2_rn(yl[p], ly));
                }
                const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                if (SELF) {
                    inv.x = (j == jself0 + (2 * p) * rstride) ? 0.f : inv.x;
                    inv.y = (j == jself0 + (2 * p + 1) * rstride) ? 0.f : inv.y;
                }
                if (WANT_E) et[p] = __fadd2_rn(et[p], inv);
                if (WANT_G) {
                    const float2 inv3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
                    gxt[p] = __ffma2_rn(dx, inv3, gxt[p]);
                    gyt[p] = __ffma2_rn(dy, inv3, gyt[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PA; ++p) {
            const float ev[2] = {et[p].x, et[p].y}, gxv[2] = {gxt[p].x, gxt[p].y}, gyv[2] = {gyt[p].x, gyt[p].y};
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int r = 2 * p + h2;
                float* a = acc + tid;
                if (WANT_E) {
                    float hi_ = a[(6 * r + 0) * stride], lo_ = a[(6 * r + 1) * stride];
                    df_add(hi_, lo_, ev[h2] * escale);
                    a[(6 * r + 0) * stride] = hi_;
                    a[(6 * r + 1) * stride] = lo_;
                }
                if (WANT_G) {
                    // the tile sums hold sum dx r^-3 = -dE/dx
                    float gh = a[(6 * r + 2) * stride], gl = a[(6 * r + 3) * stride];
                    df_add(gh, gl, -gxv[h2]);
                    a[(6 * r + 2) * stride] = gh;
                    a[(6 * r + 3) * stride] = gl;
                    float yh_ = a[(6 * r + 4) * stride], yl_ = a[(6 * r + 5) * stride];
                    df_add(yh_, yl_, -gyv[h2]);
                    a[(6 * r + 4) * stride] = yh_;
                    a[(6 * r + 5) * stride] = yl_;
                }
            }
        }
    }
};

// Warp-level min/max of a box.
__device__ __forceinline__ float4 warp_box(float4 b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b.x = fminf(b.x, __shfl_xor_sync(0xffffffffu, b.x, o));
        b.y = fminf(b.y, __shfl_xor_sync(0xffffffffu, b.y, o));
        b.z = fmaxf(b.z, __shfl_xor_sync(0xffffffffu, b.z, o));
        b.w = fmaxf(b.w, __shfl_xor_sync(0xffffffffu, b.w, o));
    }
    return b;
}

__device__ __forceinline__ float4 box_union(float4 a, float4 b)
{
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

// True when every point of box a is at least kFarDist from every point of box b.
__device__ __forceinline__ bool boxes_far(float4 a, float4 b)
{
    const float gx = fmaxf(0.f, fmaxf(a.x - b.z, b.x - a.z));
    const float gy = fmaxf(0.f, fmaxf(a.y - b.w, b.y - a.w));
    return gx * gx + gy * gy >= kFarDist * kFarDist;
}

// The mixed pass kernel.  THREADS threads per CTA, R rows per thread (row
// block RB = THREADS * R), tiles of T sources (T / THREADS staged per thread);
// MINB: resident CTAs per SM the register allocation must allow.  The next
// tile's sources arrive by cp.async in a landing buffer while the current tile
// is computed; the problem record, boxes, lo parts and accumulators live in
// shared memory.
template <int R, int THREADS, int T, int MINB, bool WANT_E, bool WANT_G>
__global__ void __launch_bounds__(THREADS, MINB) k_pass_mixed(PassArgs a, int64_t u_base, int64_t row_sub)
{
    static_assert(T % THREADS == 0, "each thread stages a whole number of sources");
    constexpr int S = T / THREADS;
    constexpr int RB = THREADS * R;
    constexpr int NW = THREADS / 32;
    constexpr int P = R / 2;
    __shared__ float4 shi[2][T];
    __shared__ float4 slo[2][T];
    __shared__ float4 sraw[T];
    __shared__ float4 swbox[2][NW];
    __shared__ float4 srbox[NW];
    __shared__ float sacc[6 * R * THREADS];
    __shared__ float2 slo2[4 * P * THREADS];
    __shared__ Prob sprob;
    __shared__ int sprob_s;

    __shared__ unsigned sticket;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // ranges: one per CTA, or (a.ticket) a.ranges of them taken in order from the ticket counter;
    // a range's slots depend on the range alone, so no result depends on which CTA takes it
    const int64_t G = a.ticket ? a.ranges : gridDim.x;
    int64_t k = blockIdx.x;

    MixedRows<R> rs;
    unsigned valid = 0;  // bit c: this thread's c-th staged source is a real charge
    // start the copies of tile t's sources (positions tid + c * THREADS) into sraw
    auto fetch = [&](int t) {
        valid = 0;
#pragma unroll
        for (int c = 0; c < S; ++c) {
            const int jt = tid + c * THREADS;
            const float4* src;
            bool ok;
            if (t < sprob.n_t_snap) {
                const int64_t j = (int64_t)t * T + jt;
                ok = j < sprob.snap_e - sprob.snap_b;
                if (ok && sprob.mask_off >= 0) ok = ((a.mask[sprob.mask_off + (j >> 5)] >> (j & 31)) & 1u) == 0u;
                src = static_cast<const float4*>(a.snap) + sprob.snap_b + j;
            } else {
                const int64_t j = (int64_t)(t - sprob.n_t_snap) * T + jt;
                ok = j < sprob.m;
                src = static_cast<const float4*>(a.rows) + sprob.row_base + j;
            }
            if (ok) {
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sraw[jt]);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
                valid |= 1u << c;
            } else {
                sraw[jt] = make_float4(kFar32, kFar32, 0.f, 0.f);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    // wait for them and stage into buffer b (negated hi/lo lanes) with the warp's box
    auto stage = [&](int b) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        float4 bx = make_float4(kBoxEmptyLo, kBoxEmptyLo, kBoxEmptyHi, kBoxEmptyHi);
#pragma unroll
        for (int c = 0; c < S; ++c) {
            const int jt = tid + c * THREADS;
            const float4 q = sraw[jt];
            shi[b][jt] = make_float4(-q.x, -q.x, -q.y, -q.y);
            slo[b][jt] = make_float4(-q.z, -q.z, -q.w, -q.w);
            if ((valid >> c) & 1u) bx = box_union(bx, make_float4(q.x, q.y, q.x, q.y));
        }
        bx = warp_box(bx);
        if (lane == 0) swbox[b][warp] = bx;
    };
    for (;;) {
    if (a.ticket) {
        if (tid == 0) sticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        k = sticket;
        __syncthreads();
        if (k >= G) {
            // every CTA draws exactly one ticket >= G; the last of them is drawn last
            if (tid == 0 && k == G + gridDim.x - 1) *a.ticket = 0u;
            break;
        }
    }
    int64_t u = sk_begin(a.W, G, k);
    const int64_t u_end = sk_begin(a.W, G, k + 1);
    while (u < u_end) {
        if (tid == 0) {
            const int s = a.prob ? find_prob(a.prob, a.S, u_base + u) : 0;
            sprob = a.prob ? a.prob[s] : a.single;
            sprob_s = s;
        }
        __syncthreads();
        const int n_t = sprob.n_t_snap + sprob.n_t_priv;
        const int64_t local = u_base + u - sprob.unit_off;
        const int rb = (int)(local / n_t);
        const int t0 = (int)(local % n_t);
        const int t1 = (int)min((int64_t)n_t, (int64_t)t0 + (u_end - u));
        const bool act = (a.active == nullptr) || (a.active[sprob_s] != 0);
        if (act) {
            // A partial last row block: when its rows fit in the first PH
            // pairs of every thread (rows tid + r * THREADS), all warps compute
            // those pairs only (`half`); otherwise its rows go to the first
            // rstride threads (rstride a multiple of 32, rows tid + r * rstride)
            // and whole warps that hold no row skip the tile arithmetic.
            // Halving every warp's work keeps the SM's schedulers evenly loaded,
            // which idle warps do not.
            constexpr int PH = P >= 2 ? P / 2 : P;
            const int m_blk = (int)min((int64_t)RB, (int64_t)sprob.m - (int64_t)rb * RB);
            const bool half = P >= 2 && m_blk <= 2 * PH * THREADS;
            const int rstride = half ? THREADS : min(THREADS, (((m_blk + R - 1) / R) + 31) & ~31);
            const bool holds = tid < rstride;
            const int64_t rl0 = (int64_t)rb * RB + tid;
            float4 rbox = warp_box(rs.load(static_cast<const float4*>(a.rows), sprob.row_base, rl0, rstride, holds,
                                           sprob.m, slo2, sacc, THREADS, tid));
            if (lane == 0) srbox[warp] = rbox;
            fetch(t0);
            stage(0);
            __syncthreads();
            for (int t = t0; t < t1; ++t) {
                const int buf = (t - t0) & 1;
                if (t + 1 < t1) fetch(t + 1);
                float4 tbox = swbox[buf][0], rb4 = srbox[0];
#pragma unroll
                for (int w = 1; w < NW; ++w) {
                    tbox = box_union(tbox, swbox[buf][w]);
                    rb4 = box_union(rb4, srbox[w]);
                }
                const bool own = t >= sprob.n_t_snap;
                const int tp = t - sprob.n_t_snap;
                const bool self = own && (rb * RB < tp * T + T) && (tp * T < rb * RB + RB);
                const int jself0 = (int)(rl0 - (int64_t)tp * T);
                const float sc = own ? 0.5f : 1.0f;
                // each buffer gets its own copy of the tile loop, so the shared
                // memory base is a compile-time address and every source load
                // uses an immediate offset
                const int kind = self ? 2 : (boxes_far(rb4, tbox) ? 0 : 1);
                if (holds) {
                    if (buf == 0) {
                        if (kind == 0 && half)
                            rs.template tile<T, false, false, WANT_E, WANT_G, PH>(shi[0], slo[0], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else if (kind == 0)
                            rs.template tile<T, false, false, WANT_E, WANT_G>(shi[0], slo[0], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else if (kind == 1)
                            rs.template tile<T, true, false, WANT_E, WANT_G>(shi[0], slo[0], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else
                            rs.template tile<T, true, true, WANT_E, WANT_G>(shi[0], slo[0], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                    } else {
                        if (kind == 0 && half)
                            rs.template tile<T, false, false, WANT_E, WANT_G, PH>(shi[1], slo[1], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else if (kind == 0)
                            rs.template tile<T, false, false, WANT_E, WANT_G>(shi[1], slo[1], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else if (kind == 1)
                            rs.template tile<T, true, false, WANT_E, WANT_G>(shi[1], slo[1], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                        else
                            rs.template tile<T, true, true, WANT_E, WANT_G>(shi[1], slo[1], slo2, sacc, THREADS, tid, jself0, rstride, sc);
                    }
                }
                if (t + 1 < t1) stage(buf ^ 1);
                __syncthreads();
            }
            const int64_t slot = k - sk_owner(sprob.unit_off + (int64_t)rb * n_t - u_base, a.W, G);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t rl = rl0 + (int64_t)r * rstride;
                if (holds && rl < sprob.m) {
                    const int64_t o = slot * a.M + sprob.row_base + rl - row_sub;
                    const float* ac = sacc + tid;
                    if (WANT_E) a.part_e[o] = (double)ac[(6 * r + 0) * THREADS] + (double)ac[(6 * r + 1) * THREADS];
                    if (WANT_G)
                        a.part_g[o] = make_double2((double)ac[(6 * r + 2) * THREADS] + (double)ac[(6 * r + 3) * THREADS],
                                                   (double)ac[(6 * r + 4) * THREADS] + (double)ac[(6 * r + 5) * THREADS]);
                }
            }
        }
        u += t1 - t0;
        __syncthreads();  // every thread is done with sprob before the next segment rewrites it
    }
    if (!a.ticket) break;
    }
}

}  // namespace tc
