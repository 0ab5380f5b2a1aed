// tc_pass.cuh -- the generic pair pass: persistent CTAs, stream-K unit split,
// source tiles staged in shared memory, per-row partial sums out.
//
// Unit = (one row block of RB = THREADS*R moving charges) x (one tile of
// T = THREADS sources).  A CTA walks its contiguous unit range; every time it
// leaves a row block it writes that block's partial row sums to the slot
// (its CTA index minus the index of the first CTA touching the block), so the
// reducer can add the slots of a row in a fixed order (deterministic).
#pragma once

#include <type_traits>

#include "tc_device.cuh"

namespace tc {

// Rows of one thread and their accumulators, per pass flavour (the float32
// pass has its own kernel, tc_pass_mixed.cuh).
template <int KIND, int R> struct RowState;

// ---- float64 pair terms --------------------------------------------------------
template <int R> struct RowState<PASS_F64, R> {
    double x[R], y[R];
    double eh[R], el[R], gx[R], gy[R];

    __device__ void load(const double2* rows, int64_t base, int64_t rl0, int stride, int m)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t rl = rl0 + (int64_t)r * stride;
            double2 q = (rl < m) ? rows[base + rl] : make_double2(kFarRow64, kFarRow64);
            x[r] = q.x; y[r] = q.y;
            eh[r] = el[r] = gx[r] = gy[r] = 0.0;
        }
    }

    template <int T, bool SELF, bool WANT_E, bool WANT_G>
    __device__ __forceinline__ void tile(const double2* __restrict__ s, const int (&jself)[R], double escale)
    {
        double et[R];
#pragma unroll
        for (int r = 0; r < R; ++r) et[r] = 0.0;
#pragma unroll 2
        for (int j = 0; j < T; ++j) {
            const double2 q = s[j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double dx = x[r] - q.x;
                double dy = y[r] - q.y;
                double r2 = fma(dx, dx, dy * dy);
                double inv = rsqrt64(r2);
                if (SELF) inv = (j == jself[r]) ? 0.0 : inv;
                if (WANT_E) et[r] += inv;
                if (WANT_G) {
                    double inv3 = inv * inv * inv;
                    gx[r] = fma(-dx, inv3, gx[r]);
                    gy[r] = fma(-dy, inv3, gy[r]);
                }
            }
        }
        if (WANT_E) {
#pragma unroll
            for (int r = 0; r < R; ++r) dd_add(eh[r], el[r], et[r] * escale);
        }
    }

    // One chunk of 32 sources that lie after the row block, each unordered pair
    // once: lane l pairs its rows with source (l + k) mod 32 at step k, adds the
    // terms to its rows (as tile()) and the opposite gradient and the same
    // 1/r to the source's sums (ax, ay, ae), and then takes lane l + 1's source
    // sums, which belong to its next source.  After the 32 steps lane l holds
    // the sums of source l of the chunk (over this warp's rows).  et collects
    // the rows' 1/r sums of the tile.
    template <bool WANT_E, bool WANT_G>
    __device__ __forceinline__ void chunk_sym(const double2* __restrict__ s, double& ax, double& ay, double& ae,
                                              double (&et)[R])
    {
        const int lane = threadIdx.x & 31;
        const int next = (lane + 1) & 31;
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const double2 q = s[(lane + k) & 31];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const double dx = x[r] - q.x;
                const double dy = y[r] - q.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double inv = rsqrt64(r2);
                if (WANT_E) {
                    et[r] += inv;
                    ae += inv;
                }
                if (WANT_G) {
                    const double inv3 = inv * inv * inv;
                    gx[r] = fma(-dx, inv3, gx[r]);
                    gy[r] = fma(-dy, inv3, gy[r]);
                    ax = fma(dx, inv3, ax);
                    ay = fma(dy, inv3, ay);
                }
            }
            if (WANT_G) {
                ax = __shfl_sync(0xffffffffu, ax, next);
                ay = __shfl_sync(0xffffffffu, ay, next);
            }
            if (WANT_E) ae = __shfl_sync(0xffffffffu, ae, next);
        }
    }

    template <bool WANT_E> __device__ __forceinline__ void add_energy(const double (&et)[R], double escale)
    {
        if (WANT_E) {
#pragma unroll
            for (int r = 0; r < R; ++r) dd_add(eh[r], el[r], et[r] * escale);
        }
    }

    __device__ double e(int r) const { return eh[r] + el[r]; }
    __device__ double2 g(int r) const { return make_double2(gx[r], gy[r]); }
};

// ---- float64 pairwise energy change: rows and own-row sources carry (old, new) -----
template <int R> struct RowState<PASS_DELTA, R> {
    double ox[R], oy[R], nx[R], ny[R];
    double dh[R], dl[R];

    __device__ void load(const d4* rows, int64_t base, int64_t rl0, int stride, int m)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t rl = rl0 + (int64_t)r * stride;
            d4 q = (rl < m) ? rows[base + rl] : make_d4(kFarRow64, kFarRow64, kFarRow64, kFarRow64);
            ox[r] = q.x; oy[r] = q.y; nx[r] = q.z; ny[r] = q.w;
            dh[r] = dl[r] = 0.0;
        }
    }

    // OWN = false: snapshot sources (x, y in .x, .y): term 1/|new - c| - 1/|old - c|.
    // OWN = true: own rows (old, new): term 1/|new - new'| - 1/|old - old'|.
    template <int T, bool SELF, bool OWN>
    __device__ __forceinline__ void tile(const d4* __restrict__ s, const int (&jself)[R], double escale)
    {
        double dt[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dt[r] = 0.0;
#pragma unroll 2
        for (int j = 0; j < T; ++j) {
            const d4 q = s[j];
            const double sx1 = OWN ? q.z : q.x, sy1 = OWN ? q.w : q.y;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double ax = nx[r] - sx1, ay = ny[r] - sy1;
                double bx = ox[r] - q.x, by = oy[r] - q.y;
                double inv1 = rsqrt64(fma(ax, ax, ay * ay));
                double inv0 = rsqrt64(fma(bx, bx, by * by));
                double d = inv1 - inv0;
                if (SELF) d = (j == jself[r]) ? 0.0 : d;
                dt[r] += d;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) dd_add(dh[r], dl[r], dt[r] * escale);
    }

    __device__ double e(int r) const { return dh[r] + dl[r]; }
};

// ---- difference-form energy change in float32 (rows and own sources carry a move) ----
// For a pair with old separation d and move m of the separation (the row's move
// minus the source's), the new separation is d' = d + m and
//     1/|d'| - 1/|d| = (|d|^2 - |d'|^2) / (|d| |d'| (|d| + |d'|)),
//     |d|^2 - |d'|^2 = -m . (d + d'),
// which stays accurate relative to the move instead of cancelling two 1/r terms.
// Alongside it accumulates b = |m|_a / |d'| (1/|d| + 1/|d'|), |m|_a the L1 norm of
// the moves entering m (the row's, plus the source's for own rows).  b bounds
// |term| <= |m| / (|d| |d'|) and the first-order effect of float32 errors in d
// (|grad(1/|d'|) - grad(1/|d|)| <= |m| (|d| + |d'|) / (|d|^2 |d'|^2), times
// |error of d| <= 2^-22 |d|) and in m (|error of m| / |d'|^2 <= 2^-23 |m|_a / |d'|^2),
// so sum(b) scales the error bound of the float32 evaluation.
template <int R> struct RowState<PASS_DMIX, R> {
    float xh[R], yh[R], xl[R], yl[R], mx[R], my[R];
    float dh[R], dl[R], bs[R];

    __device__ void load(const f8* rows, int64_t base, int64_t rl0, int stride, int m)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t rl = rl0 + (int64_t)r * stride;
            f8 q = (rl < m) ? rows[base + rl] : make_f8(make_float4(kFarRow32, kFarRow32, 0.f, 0.f), 0.f, 0.f);
            xh[r] = q.p.x; yh[r] = q.p.y; xl[r] = q.p.z; yl[r] = q.p.w;
            mx[r] = q.d.x; my[r] = q.d.y;
            dh[r] = dl[r] = bs[r] = 0.f;
        }
    }

    // OWN = false: snapshot sources (they stay); OWN = true: own rows (they move too).
    template <int T, bool SELF, bool OWN>
    __device__ __forceinline__ void tile(const f8* __restrict__ s, const int (&jself)[R], float escale)
    {
        float dt[R], bt[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dt[r] = bt[r] = 0.f;
#pragma unroll 4
        for (int j = 0; j < T; ++j) {
            const f8 q = s[j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dx = (xh[r] - q.p.x) + (xl[r] - q.p.z);
                const float dy = (yh[r] - q.p.y) + (yl[r] - q.p.w);
                const float ux = OWN ? mx[r] - q.d.x : mx[r];
                const float uy = OWN ? my[r] - q.d.y : my[r];
                const float px = dx + ux, py = dy + uy;
                const float r2 = fmaf(dx, dx, dy * dy), r2n = fmaf(px, px, py * py);
                const float i0 = rsqrt_mufu(r2), i1 = rsqrt_mufu(r2n);
                const float num = -fmaf(ux, dx + px, uy * (dy + py));
                const float q01 = i0 * i1;
                float t = num * q01 * rcp_mufu(fmaf(r2, i0, r2n * i1));
                const float ua = OWN ? (fabsf(mx[r]) + fabsf(my[r])) + (fabsf(q.d.x) + fabsf(q.d.y))
                                     : fabsf(mx[r]) + fabsf(my[r]);
                float b = ua * (i1 * (i0 + i1));
                if (SELF) {
                    t = (j == jself[r]) ? 0.f : t;
                    b = (j == jself[r]) ? 0.f : b;
                }
                dt[r] += t;
                bt[r] += b;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            df_add(dh[r], dl[r], dt[r] * escale);
            bs[r] += bt[r] * escale;
        }
    }

    __device__ double e(int r) const { return (double)dh[r] + (double)dl[r]; }
    __device__ double bound(int r) const { return (double)bs[r]; }
};

// ---- float64-grade pair terms from float32 arithmetic ---------------------------
// Positions come as three-part float32 splits (fx3): the hi and mid differences
// are exact, so each separation is formed as a double-float (a, b) with
// |b| <= 2^-23 |a| and error ~2^-69.  r^2, 1/r (a MUFU.RSQ seed y0 and one
// correction step y = y0 + y0 (e/2 + 3e^2/8), e = 1 - r^2 y0^2 evaluated in
// double-float), r^-3 = y^3 and dx r^-3 follow in double-float (TwoProd via
// fma); each term is accurate to ~2^-46 relative.  Sums run in double-float
// (TwoSum) over chunks of 16 sources and are folded into float64 row sums.
__device__ __forceinline__ void df_acc(float& h, float& l, float vh, float vl)
{
    const float s = h + vh;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (vh - bb);
    h = s;
    l += err + vl;
}

template <int R> struct RowState<PASS_F64X, R> {
    float hx[R], hy[R], mx[R], my[R], lx[R], ly[R];
    double es[R], gs_x[R], gs_y[R];

    __device__ void load(const fx3* rows, int64_t base, int64_t rl0, int stride, int m)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t rl = rl0 + (int64_t)r * stride;
            fx3 q = (rl < m) ? rows[base + rl] : far3(kFarRow32);
            hx[r] = q.hm.x; hy[r] = q.hm.y; mx[r] = q.hm.z; my[r] = q.hm.w; lx[r] = q.lo.x; ly[r] = q.lo.y;
            es[r] = gs_x[r] = gs_y[r] = 0.0;
        }
    }

    // Sources go in chunks of kChunk: each chunk is summed in double-float and
    // folded into the float64 row sums, so no double-float sum runs over more
    // than kChunk terms (a double-float sum of n terms drifts by ~sqrt(n) 2^-48
    // of its value; over a 256-source tile that reached 1e-13 of a row's energy).
    static constexpr int kChunk = 16;

    template <int T, bool SELF, bool WANT_E, bool WANT_G>
    __device__ __forceinline__ void tile(const fx3* __restrict__ s, const int (&jself)[R], double escale)
    {
        static_assert(T % kChunk == 0, "whole chunks per tile");
#pragma unroll 1
        for (int j0 = 0; j0 < T; j0 += kChunk) {
        float eh[R], el[R], xh[R], xl[R], yh[R], yl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) eh[r] = el[r] = xh[r] = xl[r] = yh[r] = yl[r] = 0.f;
#pragma unroll 2
        for (int j = j0; j < j0 + kChunk; ++j) {
            const fx3 q = s[j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // separation (ax + bx, ay + by): exact hi and mid differences, Fast2Sum
                const float dhx = hx[r] - q.hm.x, dmx = mx[r] - q.hm.z;
                const float ax = dhx + dmx, bx = (dmx - (ax - dhx)) + (lx[r] - q.lo.x);
                const float dhy = hy[r] - q.hm.y, dmy = my[r] - q.hm.w;
                const float ay = dhy + dmy, by = (dmy - (ay - dhy)) + (ly[r] - q.lo.y);
                // r^2 = R2 + R2l
                const float p1 = ax * ax;
                float e1 = fmaf(ax, ax, -p1);
                e1 = fmaf(ax + ax, bx, e1);
                e1 = fmaf(bx, bx, e1);
                const float p2 = ay * ay;
                float e2 = fmaf(ay, ay, -p2);
                e2 = fmaf(ay + ay, by, e2);
                e2 = fmaf(by, by, e2);
                const float R2 = p1 + p2;
                const float bb = R2 - p1;
                const float R2l = ((p1 - (R2 - bb)) + (p2 - bb)) + (e1 + e2);
                // 1/r = y0 + c
                float y0 = rsqrt_mufu(R2);
                if (SELF) y0 = (j == jself[r]) ? 0.f : y0;
                const float th = y0 * y0, tl = fmaf(y0, y0, -th);
                const float qh = R2 * th;
                float ql = fmaf(R2, th, -qh);
                ql = fmaf(R2, tl, ql);
                ql = fmaf(R2l, th, ql);
                const float ee = (1.f - qh) - ql;
                const float c = y0 * (ee * fmaf(0.375f, ee, 0.5f));
                if (WANT_E) df_acc(eh[r], el[r], y0, c);
                if (WANT_G) {
                    // r^-3 = y^3 = (th + sl) y
                    float sl = fmaf(y0 + y0, c, tl);
                    sl = fmaf(c, c, sl);
                    const float uh = th * y0;
                    float ul = fmaf(th, y0, -uh);
                    ul = fmaf(th, c, ul);
                    ul = fmaf(sl, y0, ul);
                    const float gxh = ax * uh;
                    float gxl = fmaf(ax, uh, -gxh);
                    gxl = fmaf(ax, ul, gxl);
                    gxl = fmaf(bx, uh, gxl);
                    const float gyh = ay * uh;
                    float gyl = fmaf(ay, uh, -gyh);
                    gyl = fmaf(ay, ul, gyl);
                    gyl = fmaf(by, uh, gyl);
                    df_acc(xh[r], xl[r], gxh, gxl);
                    df_acc(yh[r], yl[r], gyh, gyl);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (WANT_E) es[r] += ((double)eh[r] + (double)el[r]) * escale;
            if (WANT_G) {
                gs_x[r] -= (double)xh[r] + (double)xl[r];
                gs_y[r] -= (double)yh[r] + (double)yl[r];
            }
        }
        }
    }

    __device__ double e(int r) const { return es[r]; }
    __device__ double2 g(int r) const { return make_double2(gs_x[r], gs_y[r]); }
};

// Source entry t*T + tid of a problem's tile list, with masking and padding.
template <int KIND, int T>
__device__ __forceinline__ typename SrcT<KIND>::type load_src(const PassArgs& a, const Prob& p, int t, int tid)
{
    using src_t = typename SrcT<KIND>::type;
    if (t < p.n_t_snap) {
        int64_t j = (int64_t)t * T + tid;
        bool ok = j < p.snap_e - p.snap_b;
        if (ok && p.mask_off >= 0) {
            uint32_t w = a.mask[p.mask_off + (j >> 5)];
            ok = ((w >> (j & 31)) & 1u) == 0u;
        }
        if constexpr (KIND == PASS_DMIX) {
            return make_f8(ok ? static_cast<const float4*>(a.snap)[p.snap_b + j] : make_float4(kFar32, kFar32, 0.f, 0.f),
                           0.f, 0.f);
        } else if constexpr (KIND == PASS_F64X) {
            return ok ? static_cast<const fx3*>(a.snap)[p.snap_b + j] : far3(kFar32);
        } else if constexpr (KIND == PASS_F64) {
            return ok ? static_cast<const double2*>(a.snap)[p.snap_b + j] : make_double2(kFar64, kFar64);
        } else {
            double2 c = ok ? static_cast<const double2*>(a.snap)[p.snap_b + j] : make_double2(kFar64, kFar64);
            return make_d4(c.x, c.y, c.x, c.y);
        }
    } else {
        int64_t j = (int64_t)(t - p.n_t_snap) * T + tid;
        bool ok = j < p.m;
        if constexpr (KIND == PASS_DMIX) {
            return ok ? static_cast<const f8*>(a.rows)[p.row_base + j]
                      : make_f8(make_float4(kFar32, kFar32, 0.f, 0.f), 0.f, 0.f);
        } else if constexpr (KIND == PASS_F64X) {
            return ok ? static_cast<const fx3*>(a.rows)[p.row_base + j] : far3(kFar32);
        } else if constexpr (KIND == PASS_F64) {
            return ok ? static_cast<const double2*>(a.rows)[p.row_base + j] : make_double2(kFar64, kFar64);
        } else {
            return ok ? static_cast<const d4*>(a.rows)[p.row_base + j]
                      : make_d4(kFar64, kFar64, kFar64, kFar64);
        }
    }
}

// The pass.  Grid: persistent CTAs (any count); each takes units
// [u_base + b_k, u_base + b_{k+1}) of the W units starting at u_base, or (a.ticket)
// the ranges k drawn from the ticket counter.  Row partials go to
// part_e/part_g[slot * M + row - row_sub]; with a.sym (float64), source sums of
// the later tiles go to col_e/col_g (PassArgs).
template <int KIND, int R, int THREADS, bool WANT_E, bool WANT_G, bool SYM = false>
__global__ void __launch_bounds__(THREADS) k_pass(PassArgs a, int64_t u_base, int64_t row_sub)
{
    constexpr int T = THREADS;
    constexpr int RB = THREADS * R;
    constexpr int NW = THREADS / 32;
    using src_t = typename SrcT<KIND>::type;  // rows use the same entry type as sources
    __shared__ src_t tile[2][T];
    constexpr bool SYM_OK = SYM && KIND == PASS_F64 && RB == 2 * T;
    __shared__ double csum[SYM_OK ? 3 : 1][SYM_OK ? NW : 1][32];  // per warp: a chunk's source sums
    __shared__ unsigned sticket;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t G = a.ticket ? a.ranges : gridDim.x;
    int64_t k = blockIdx.x;

    RowState<KIND, R> rs;
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
        const int s = a.prob ? find_prob(a.prob, a.S, u_base + u) : 0;
        const Prob p = a.prob ? a.prob[s] : a.single;
        const int n_t = p.n_t_snap + p.n_t_priv;
        const int64_t local = u_base + u - p.unit_off;
        const int rb = (int)(local / n_t);
        const int t1 = (int)min((int64_t)n_t, (int64_t)(local % n_t) + (u_end - u));
        const int tu = (int)(local % n_t);  // the segment's first unit
        // symmetric float64 pass: the tiles before the row block's own ones do nothing
        const bool sym = SYM_OK && a.sym;
        const int t0 = sym ? max(tu, 2 * rb) : tu;
        const bool act = (a.active == nullptr) || (a.active[s] != 0);
        if (act) {
            // A partial last row block gives its rows to the first rstride
            // threads (rstride a multiple of 32, rows tid + r * rstride), so
            // whole warps hold no row and skip the pair arithmetic.
            const int m_blk = (int)min((int64_t)RB, (int64_t)p.m - (int64_t)rb * RB);
            const int rstride = min(THREADS, (((m_blk + R - 1) / R) + 31) & ~31);
            const bool holds = tid < rstride;
            const int64_t rl0 = (int64_t)rb * RB + tid;
            rs.load(static_cast<const src_t*>(a.rows), p.row_base, rl0, rstride, holds ? p.m : 0);
            src_t pre{};
            if (t0 < t1) {
                pre = load_src<KIND, T>(a, p, t0, tid);
                tile[0][tid] = pre;
            }
            __syncthreads();
            for (int t = t0; t < t1; ++t) {
                const int buf = (t - t0) & 1;
                if (t + 1 < t1) pre = load_src<KIND, T>(a, p, t + 1, tid);
                const bool own = t >= p.n_t_snap;
                const int tp = t - p.n_t_snap;
                const bool self = own && (rb * RB < tp * T + T) && (tp * T < rb * RB + RB);
                int jself[R];
#pragma unroll
                for (int r = 0; r < R; ++r) jself[r] = (int)(rl0 + r * rstride) - tp * T;
                const double sc = own ? 0.5 : 1.0;
                if constexpr (KIND == PASS_DELTA || KIND == PASS_DMIX) {
                    using sc_t = typename std::conditional<KIND == PASS_DELTA, double, float>::type;
                    if (!holds) {
                    } else if (!own)
                        rs.template tile<T, false, false>(tile[buf], jself, (sc_t)sc);
                    else if (self)
                        rs.template tile<T, true, true>(tile[buf], jself, (sc_t)sc);
                    else
                        rs.template tile<T, false, true>(tile[buf], jself, (sc_t)sc);
                } else if constexpr (SYM_OK) {
                    if (sym && tp >= 2 * rb + 2) {
                        // a later tile: each pair once, the source sums per chunk of 32 sources
                        double et[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) et[r] = 0.0;
                        for (int c = 0; c < T / 32; ++c) {
                            double ax = 0.0, ay = 0.0, ae = 0.0;
                            if (holds) rs.template chunk_sym<WANT_E, WANT_G>(tile[buf] + c * 32, ax, ay, ae, et);
                            csum[0][warp][lane] = ax;
                            csum[1][warp][lane] = ay;
                            csum[2][warp][lane] = ae;
                            __syncthreads();
                            if (tid < 32) {
                                double sx = 0.0, sy = 0.0, se = 0.0;
#pragma unroll
                                for (int w = 0; w < NW; ++w) {
                                    sx += csum[0][w][tid];
                                    sy += csum[1][w][tid];
                                    se += csum[2][w][tid];
                                }
                                const int64_t j = (int64_t)tp * T + c * 32 + tid;
                                if (j < p.m) {
                                    const int64_t o = (int64_t)rb * a.col_stride + p.row_base + j - row_sub;
                                    if (WANT_E) a.col_e[o] = se * sc;
                                    if (WANT_G) a.col_g[o] = make_double2(sx, sy);
                                }
                            }
                            __syncthreads();
                        }
                        rs.template add_energy<WANT_E>(et, sc);
                    } else if (!holds) {
                    } else if (self) {
                        rs.template tile<T, true, WANT_E, WANT_G>(tile[buf], jself, sc);
                    } else {
                        rs.template tile<T, false, WANT_E, WANT_G>(tile[buf], jself, sc);
                    }
                } else {
                    if (!holds) {
                    } else if (self)
                        rs.template tile<T, true, WANT_E, WANT_G>(tile[buf], jself, (float)sc);
                    else
                        rs.template tile<T, false, WANT_E, WANT_G>(tile[buf], jself, (float)sc);
                }
                if (t + 1 < t1) tile[buf ^ 1][tid] = pre;
                __syncthreads();
            }
            const int64_t slot = k - sk_owner(p.unit_off + (int64_t)rb * n_t - u_base, a.W, G);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t rl = rl0 + (int64_t)r * rstride;
                if (holds && rl < p.m) {
                    const int64_t o = slot * a.M + p.row_base + rl - row_sub;
                    if (WANT_E || KIND == PASS_DELTA || KIND == PASS_DMIX) a.part_e[o] = rs.e(r);
                    if constexpr (KIND == PASS_DMIX) {
                        if (a.part_g) a.part_g[o] = make_double2(rs.bound(r), 0.0);
                    } else if constexpr (KIND != PASS_DELTA) {
                        if (WANT_G) a.part_g[o] = rs.g(r);
                    }
                }
            }
        }
        u += t1 - tu;
        __syncthreads();  // the next segment's first tile overwrites tile[0]
    }
    if (!a.ticket) break;
    }
}

}  // namespace tc
