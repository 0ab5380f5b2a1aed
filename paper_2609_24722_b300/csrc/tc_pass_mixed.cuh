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

// Packed rows of one thread: R rows as R/2 float2 pairs.
template <int R> struct MixedRows {
    static_assert(R % 2 == 0, "rows come in pairs");
    static constexpr int P = R / 2;
    float2 xh[P], yh[P], xl[P], yl[P];
    float eh[R], el[R], gxh[R], gxl[R], gyh[R], gyl[R];

    // Loads rows rl0 + r*stride (r < R); rows past m sit far away.  Returns
    // the bounding box (xmin, ymin, xmax, ymax) of the valid rows' hi parts.
    __device__ float4 load(const float4* rows, int64_t base, int64_t rl0, int stride, int m)
    {
        float4 box = make_float4(kBoxEmptyLo, kBoxEmptyLo, kBoxEmptyHi, kBoxEmptyHi);
        float4 q[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t rl = rl0 + (int64_t)r * stride;
            const bool ok = rl < m;
            q[r] = ok ? rows[base + rl] : make_float4(kFarRow32, kFarRow32, 0.f, 0.f);
            if (ok) {
                box.x = fminf(box.x, q[r].x);
                box.y = fminf(box.y, q[r].y);
                box.z = fmaxf(box.z, q[r].x);
                box.w = fmaxf(box.w, q[r].y);
            }
            eh[r] = el[r] = gxh[r] = gxl[r] = gyh[r] = gyl[r] = 0.f;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            xh[p] = make_float2(q[2 * p].x, q[2 * p + 1].x);
            yh[p] = make_float2(q[2 * p].y, q[2 * p + 1].y);
            xl[p] = make_float2(q[2 * p].z, q[2 * p + 1].z);
            yl[p] = make_float2(q[2 * p].w, q[2 * p + 1].w);
        }
        return box;
    }

    // One tile of T sources.  hi[j] = (-x_hi, -x_hi, -y_hi, -y_hi), lo[j] the
    // same for the lo parts.  Accumulates sum dx r^-3 (= -grad) and sum 1/r.
    // SCALAR_TAIL: the work after the two MUFU.RSQ results (r^-3 and the two
    // gradient fmas) runs as scalar float32 per lane instead of packed pairs,
    // so the two results never have to be gathered into one register pair.
    template <int T, bool NEAR, bool SELF, bool WANT_E, bool WANT_G, bool SCALAR_TAIL>
    __device__ __forceinline__ void tile(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                         const int (&jself)[R], float escale)
    {
        if constexpr (SCALAR_TAIL)
            tile_scalar_tail<T, NEAR, SELF, WANT_E, WANT_G>(hi, lo, jself, escale);
        else
            tile_packed<T, NEAR, SELF, WANT_E, WANT_G>(hi, lo, jself, escale);
    }

    template <int T, bool NEAR, bool SELF, bool WANT_E, bool WANT_G>
    __device__ __forceinline__ void tile_packed(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                                const int (&jself)[R], float escale)
    {
        float2 et[P], gxt[P], gyt[P];
#pragma unroll
        for (int p = 0; p < P; ++p) et[p] = gxt[p] = gyt[p] = make_float2(0.f, 0.f);
#pragma unroll 4
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
            for (int p = 0; p < P; ++p) {
                float2 dx = __fadd2_rn(xh[p], qx);
                float2 dy = __fadd2_rn(yh[p], qy);
                if (NEAR) {
                    dx = __fadd2_rn(dx, __fadd2_rn(xl[p], lx));
                    dy = __fadd2_rn(dy, __fadd2_rn(yl[p], ly));
                }
                const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                if (SELF) {
                    inv.x = (j == jself[2 * p]) ? 0.f : inv.x;
                    inv.y = (j == jself[2 * p + 1]) ? 0.f : inv.y;
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
        for (int p = 0; p < P; ++p) {
            if (WANT_E) {
                df_add(eh[2 * p], el[2 * p], et[p].x * escale);
                df_add(eh[2 * p + 1], el[2 * p + 1], et[p].y * escale);
            }
            if (WANT_G) {
                // the tile sums hold sum dx r^-3 = -dE/dx
                df_add(gxh[2 * p], gxl[2 * p], -gxt[p].x);
                df_add(gxh[2 * p + 1], gxl[2 * p + 1], -gxt[p].y);
                df_add(gyh[2 * p], gyl[2 * p], -gyt[p].x);
                df_add(gyh[2 * p + 1], gyl[2 * p + 1], -gyt[p].y);
            }
        }
    }

    template <int T, bool NEAR, bool SELF, bool WANT_E, bool WANT_G>
    __device__ __forceinline__ void tile_scalar_tail(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                                     const int (&jself)[R], float escale)
    {
        float et[R], gxt[R], gyt[R];
#pragma unroll
        for (int r = 0; r < R; ++r) et[r] = gxt[r] = gyt[r] = 0.f;
#pragma unroll 4
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
            for (int p = 0; p < P; ++p) {
                float2 dx = __fadd2_rn(xh[p], qx);
                float2 dy = __fadd2_rn(yh[p], qy);
                if (NEAR) {
                    dx = __fadd2_rn(dx, __fadd2_rn(xl[p], lx));
                    dy = __fadd2_rn(dy, __fadd2_rn(yl[p], ly));
                }
                const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                const float d0[2] = {dx.x, dx.y}, e0[2] = {dy.x, dy.y}, q0[2] = {r2.x, r2.y};
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int r = 2 * p + h2;
                    float inv = rsqrt_mufu(q0[h2]);
                    if (SELF) inv = (j == jself[r]) ? 0.f : inv;
                    if (WANT_E) et[r] += inv;
                    if (WANT_G) {
                        const float inv3 = inv * inv * inv;
                        gxt[r] = fmaf(d0[h2], inv3, gxt[r]);
                        gyt[r] = fmaf(e0[h2], inv3, gyt[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (WANT_E) df_add(eh[r], el[r], et[r] * escale);
            if (WANT_G) {
                df_add(gxh[r], gxl[r], -gxt[r]);
                df_add(gyh[r], gyl[r], -gyt[r]);
            }
        }
    }

    __device__ double e(int r) const { return (double)eh[r] + (double)el[r]; }
    __device__ double2 g(int r) const
    {
        return make_double2((double)gxh[r] + (double)gxl[r], (double)gyh[r] + (double)gyl[r]);
    }
};

// Source entry (x_hi, y_hi, x_lo, y_lo) of tile t for thread tid; `valid`
// tells whether it is a real, unmasked charge.
template <int T>
__device__ __forceinline__ float4 load_src_mixed(const PassArgs& a, const Prob& p, int t, int tid, bool& valid)
{
    if (t < p.n_t_snap) {
        int64_t j = (int64_t)t * T + tid;
        bool ok = j < p.snap_e - p.snap_b;
        if (ok && p.mask_off >= 0) {
            uint32_t w = a.mask[p.mask_off + (j >> 5)];
            ok = ((w >> (j & 31)) & 1u) == 0u;
        }
        valid = ok;
        return ok ? static_cast<const float4*>(a.snap)[p.snap_b + j] : make_float4(kFar32, kFar32, 0.f, 0.f);
    }
    int64_t j = (int64_t)(t - p.n_t_snap) * T + tid;
    valid = j < p.m;
    return valid ? static_cast<const float4*>(a.rows)[p.row_base + j] : make_float4(kFar32, kFar32, 0.f, 0.f);
}

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
// MINB: resident CTAs per SM the register allocation must allow; ST: scalar
// tail (see MixedRows::tile).
template <int R, int THREADS, int T, int MINB, bool ST, bool WANT_E, bool WANT_G>
__global__ void __launch_bounds__(THREADS, MINB) k_pass_mixed(PassArgs a, int64_t u_base, int64_t row_sub)
{
    static_assert(T % THREADS == 0, "each thread stages a whole number of sources");
    constexpr int S = T / THREADS;
    constexpr int RB = THREADS * R;
    constexpr int NW = THREADS / 32;
    __shared__ float4 shi[2][T];
    __shared__ float4 slo[2][T];
    __shared__ float4 swbox[2][NW];
    __shared__ float4 srbox[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t G = gridDim.x;
    const int64_t k = blockIdx.x;
    int64_t u = sk_begin(a.W, G, k);
    const int64_t u_end = sk_begin(a.W, G, k + 1);

    MixedRows<R> rs;
    float4 pre[S];
    bool valid[S];
    // fetch tile t's S sources of this thread (positions tid + c * THREADS)
    auto fetch = [&](const Prob& p, int t) {
#pragma unroll
        for (int c = 0; c < S; ++c) {
            bool v;
            pre[c] = load_src_mixed<T>(a, p, t, tid + c * THREADS, v);
            valid[c] = v;
        }
    };
    // stage them into buffer b (negated hi/lo lanes) with the warp's box
    auto stage = [&](int b) {
        float4 bx = make_float4(kBoxEmptyLo, kBoxEmptyLo, kBoxEmptyHi, kBoxEmptyHi);
#pragma unroll
        for (int c = 0; c < S; ++c) {
            const float4 q = pre[c];
            shi[b][tid + c * THREADS] = make_float4(-q.x, -q.x, -q.y, -q.y);
            slo[b][tid + c * THREADS] = make_float4(-q.z, -q.z, -q.w, -q.w);
            if (valid[c]) bx = box_union(bx, make_float4(q.x, q.y, q.x, q.y));
        }
        bx = warp_box(bx);
        if (lane == 0) swbox[b][warp] = bx;
    };
    while (u < u_end) {
        const int s = a.prob ? find_prob(a.prob, a.S, u_base + u) : 0;
        const Prob p = a.prob ? a.prob[s] : a.single;
        const int n_t = p.n_t_snap + p.n_t_priv;
        const int64_t local = u_base + u - p.unit_off;
        const int rb = (int)(local / n_t);
        const int t0 = (int)(local % n_t);
        const int t1 = (int)min((int64_t)n_t, (int64_t)t0 + (u_end - u));
        const bool act = (a.active == nullptr) || (a.active[s] != 0);
        if (act) {
            const int64_t rl0 = (int64_t)rb * RB + tid;
            float4 rbox = warp_box(rs.load(static_cast<const float4*>(a.rows), p.row_base, rl0, THREADS, p.m));
            if (lane == 0) srbox[warp] = rbox;
            fetch(p, t0);
            stage(0);
            __syncthreads();
            rbox = srbox[0];
#pragma unroll
            for (int w = 1; w < NW; ++w) rbox = box_union(rbox, srbox[w]);
            for (int t = t0; t < t1; ++t) {
                const int buf = (t - t0) & 1;
                if (t + 1 < t1) fetch(p, t + 1);
                float4 tbox = swbox[buf][0];
#pragma unroll
                for (int w = 1; w < NW; ++w) tbox = box_union(tbox, swbox[buf][w]);
                const bool own = t >= p.n_t_snap;
                const int tp = t - p.n_t_snap;
                const bool self = own && (rb * RB < tp * T + T) && (tp * T < rb * RB + RB);
                int jself[R];
#pragma unroll
                for (int r = 0; r < R; ++r) jself[r] = (int)(rl0 + r * THREADS) - tp * T;
                const float sc = own ? 0.5f : 1.0f;
                if (self)
                    rs.template tile<T, true, true, WANT_E, WANT_G, ST>(shi[buf], slo[buf], jself, sc);
                else if (!boxes_far(rbox, tbox))
                    rs.template tile<T, true, false, WANT_E, WANT_G, ST>(shi[buf], slo[buf], jself, sc);
                else
                    rs.template tile<T, false, false, WANT_E, WANT_G, ST>(shi[buf], slo[buf], jself, sc);
                if (t + 1 < t1) stage(buf ^ 1);
                __syncthreads();
            }
            const int64_t slot = k - sk_owner(p.unit_off + (int64_t)rb * n_t - u_base, a.W, G);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t rl = rl0 + (int64_t)r * THREADS;
                if (rl < p.m) {
                    const int64_t o = slot * a.M + p.row_base + rl - row_sub;
                    if (WANT_E) a.part_e[o] = rs.e(r);
                    if (WANT_G) a.part_g[o] = rs.g(r);
                }
            }
        }
        u += t1 - t0;
    }
}

}  // namespace tc
