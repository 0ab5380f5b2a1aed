// tc_lbfgsb.cuh -- the L-BFGS-B update (one CTA or cluster per problem).  Included by
// tc_relax.cu inside namespace tc, after the relaxation state (RelaxDev,
// SlotView, the (t, u) map and the block reductions) it uses.
#pragma once

// ------------------------------------------------------------ L-BFGS-B ---
// L-BFGS-B (Byrd, Lu, Nocedal & Zhu 1995), the optimiser of Sec. II C step 4,
// on the (t, u) variables of Sec. II D with the box t in [0, pi/2], one CTA or
// one cluster of CTAs per problem of any size (its time grows with the
// problem's rows per CTA).  A pinned
// charge's variables are (u, 0): u unbounded, the second fixed at 0.
//
// Compact representation B = theta I - W M W^T, M = K^{-1},
// K = [[-D, L^T], [L, theta S S^T]] (Byrd, Nocedal & Schnabel 1994), in padded
// coordinates of kBQ entries: entry a < kBMem is y of the a-th oldest stored
// pair, entry kBMem + a is theta s of it.  Entries of pairs not stored are 0 in
// W and the identity in K, so every sum over entries adds the non-zero terms
// in the compact order.  The products s_a.y_b, s_a.s_b and y_a.y_b are kept per
// ring slot and computed once, when the newer of the two pairs is stored.
//
// The float64 pipe is the limit (one problem runs on one SM), so the per-row
// work is kept small: rows of W are read unscaled, W' = [Y, S], and theta is
// applied to the short vectors (W = W' D, D = diag(1, theta)); W_F^T W_F is
// W^T W, known from the kept products, less the rows whose t is at a bound.

constexpr int kBMem = 8;                            // largest L-BFGS-B memory
constexpr int kBQ = 2 * kBMem;                      // padded order of K and M
constexpr int kBSmall = 3 * kBMem * kBMem + 1;      // per problem: s.y, s.s, y.y by slot, theta
constexpr int kRed = 40;                            // widest multi-value block reduction
constexpr double kHalfPi = 1.5707963267948966;      // upper bound of t

__device__ __forceinline__ void tu_bounds(bool pinned, double2& lo, double2& hi)
{
    if (pinned) {
        lo = make_double2(-INFINITY, 0.0);
        hi = make_double2(INFINITY, 0.0);
    } else {
        lo = make_double2(0.0, -INFINITY);
        hi = make_double2(kHalfPi, INFINITY);
    }
}

__device__ __forceinline__ double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Breakpoint of one variable on the path P(z - t g).
__device__ __forceinline__ double breakpoint(double z, double g, double lo, double hi)
{
    if (g < 0.0 && hi < INFINITY) return (z - hi) / g;
    if (g > 0.0 && lo > -INFINITY) return (z - lo) / g;
    return INFINITY;
}

// Warp partials of values v[OFF .. OFF + N) (N <= 32) into red[warp][OFF + i]:
// a shuffle tree per value that halves the live values at each level
// (recursive halving).  At offset o a lane keeps one half of its live values,
// sends the other half to lane ^ o and adds what it receives, so the warp
// spends about one add per value instead of five.  Every value still meets the
// other lanes' partials in the pairs and order of a shfl_down tree (an add of
// two doubles is commutative), so each partial is bit for bit that tree's.
// Value i ends in lane i << (5 - log2 NP), NP = N rounded up to a power of two.
template <int N, int OFF, int M> __device__ __forceinline__ void warp_sums(const double (&v)[M], double (*red)[kRed])
{
    static_assert(N >= 1 && N <= 32 && OFF + N <= M, "warp_sums range");
    constexpr int NP = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
    constexpr int SH = NP == 1 ? 5 : NP == 2 ? 4 : NP == 4 ? 3 : NP == 8 ? 2 : NP == 16 ? 1 : 0;
    const int lane = threadIdx.x & 31;
    double x[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) x[i] = i < N ? v[OFF + i] : 0.0;
#pragma unroll
    for (int o = 16, c = NP; o > 0; o >>= 1) {
        if (c > 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < NP / 2; ++k)
                if (k < c / 2) {
                    const double keep = up ? x[k + c / 2] : x[k], send = up ? x[k] : x[k + c / 2];
                    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            c /= 2;
        } else {
            x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
        }
    }
    const int i = lane >> SH;
    if ((lane & ((1 << SH) - 1)) == 0 && i < N) red[threadIdx.x >> 5][OFF + i] = x[0];
}

// Deterministic block sums of N doubles per thread: warp partials (warp_sums,
// 32 values at a time), then the warps' partials in warp order.
template <int N> __device__ void block_sums_w(double (&v)[N], double (*red)[kRed])
{
    static_assert(N <= kRed, "reduction too wide");
    warp_sums<(N < 32 ? N : 32), 0>(v, red);
    if constexpr (N > 32) warp_sums<N - 32, 32>(v, red);
    __syncthreads();
    if (threadIdx.x < N) {
        double t = red[0][threadIdx.x];
        for (int k = 1; k < kUpd / 32; ++k) t += red[k][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = red[0][i];
    __syncthreads();
}

// Smallest (t, row) over a warp, ties to the lower row; every lane gets it (a
// minimum with a fixed tie rule does not depend on the order of comparisons).
__device__ __forceinline__ void warp_argmin(double& t, int& r)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t2 = __shfl_xor_sync(0xffffffffu, t, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
        if (t2 < t || (t2 == t && r2 < r)) {
            t = t2;
            r = r2;
        }
    }
}

// Smallest (t, row) over the block, ties to the lower row.
__device__ void block_argmin(double& t, int& r, double* sht, int* shr)
{
    warp_argmin(t, r);
    if ((threadIdx.x & 31) == 0) {
        sht[threadIdx.x >> 5] = t;
        shr[threadIdx.x >> 5] = r;
    }
    __syncthreads();
    t = sht[0];
    r = shr[0];
    for (int w = 1; w < kUpd / 32; ++w)
        if (sht[w] < t || (sht[w] == t && shr[w] < r)) {
            t = sht[w];
            r = shr[w];
        }
    __syncthreads();
}

// Row of the largest |a[r * ld + col]| over rows col .. kBQ-1, the first such
// row on ties (as a search that keeps the first maximum), or -1 if that value
// is 0; every lane of the calling warp gets it.  For doubles that are not
// negative the order of their bit patterns as integers is their numeric order,
// so the search compares integers (a NaN entry counts as 0 and is never taken).
__device__ __forceinline__ int warp_pivot(const double* a, int ld, int col)
{
    const int r0 = threadIdx.x & 31;
    unsigned long long key = 0ull;
    if (r0 >= col && r0 < kBQ) {
        const double v = a[r0 * ld + col];
        key = v == v ? (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull : 0ull;
    }
    int r = r0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
        if (k2 > key || (k2 == key && r2 < r)) {
            key = k2;
            r = r2;
        }
    }
    return key > 0ull ? r : -1;
}

// [K | I] -> [I | K^{-1}] by Gauss-Jordan elimination with partial pivoting,
// the whole CTA taking part (two of the 16 x 32 entries per thread).  Every
// entry sees the same operations in the same order as a one-lane-per-column
// elimination.  Per column, warp 0 finds the pivot, swaps and divides the
// pivot row and records the column for the elimination (one CTA barrier), then
// every thread eliminates (a second barrier).  False (for every thread) if a
// pivot is 0.
__device__ bool block_gauss_jordan(double* aug, double* fcol, int* sh_piv)
{
    constexpr int ld = 2 * kBQ;
    static_assert(ld == 32 && kBQ * ld == 2 * kUpd, "two entries per thread");
    const int t = threadIdx.x;
    for (int col = 0; col < kBQ; ++col) {
        if (t < 32) {
            const int piv = warp_pivot(aug, ld, col);
            if (t == 0) *sh_piv = piv;
            if (piv >= 0) {
                const double pv = aug[piv * ld + col];
                const double a = aug[col * ld + t], b = aug[piv * ld + t];
                // column col of every other row once the rows are swapped
                if (t < kBQ) fcol[t] = t == piv ? aug[col * ld + col] : aug[t * ld + col];
                __syncwarp();
                if (piv != col) aug[piv * ld + t] = a;
                aug[col * ld + t] = __ddiv_rn(b, pv);
            }
        }
        __syncthreads();
        if (*sh_piv < 0) return false;
#pragma unroll
        for (int e = t; e < kBQ * ld; e += kUpd) {
            const int r = e / ld, c = e % ld;
            const double f = fcol[r];
            if (r != col && f != 0.0) aug[e] = __dsub_rn(aug[e], __dmul_rn(f, aug[col * ld + c]));
        }
        __syncthreads();
    }
    return true;
}

// Row rl's two rows of W' = [Y, S] (variables x and y) in the padded coordinates.
__device__ __forceinline__ void w_rows(const RelaxDev& d, int64_t row, const int* slot, int hb,
                                       double (&wx)[kBQ], double (&wy)[kBQ])
{
#pragma unroll
    for (int a = 0; a < kBMem; ++a) {
        if (a < hb) {
            const int j = slot[a];
            const double2 yj = d.Yh[(int64_t)j * d.M + row], sj = d.Sh[(int64_t)j * d.M + row];
            wx[a] = yj.x;
            wy[a] = yj.y;
            wx[kBMem + a] = sj.x;
            wy[kBMem + a] = sj.y;
        } else {
            wx[a] = wy[a] = wx[kBMem + a] = wy[kBMem + a] = 0.0;
        }
    }
}

__device__ __forceinline__ double dot16(const double (&w)[kBQ], const double* v)
{
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < kBQ; ++a) s += w[a] * v[a];
    return s;
}

// Row a of M x (sums in entry order); one lane per row.
__device__ __forceinline__ double row_dot16(const double* M, const double* x, int a)
{
    double s = 0.0;
    for (int b = 0; b < kBQ; ++b) s += M[a * kBQ + b] * x[b];
    return s;
}

// Sum of v over lanes 0 .. kBQ - 1 of a warp (fixed tree), valid in lane 0.
__device__ __forceinline__ double lanes_sum16(double v)
{
#pragma unroll
    for (int o = kBQ / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ---- one problem stepped by a cluster of CL CTAs ----
// The rows of a problem are dealt to the CTAs in blocks of kUpd (CTA r takes
// rows r kUpd .. r kUpd + kUpd - 1, then (r + CL) kUpd .., and so on).  A
// reduction first reduces within each CTA (every thread gets the CTA's totals),
// then each CTA posts its totals in its own shared memory, the cluster waits
// at its barrier, and every CTA adds the CL posts in rank order: all CTAs hold
// the same totals, bit for bit, and repeat the small dense algebra on them.
// Posts alternate between two buffers; a CTA writes a buffer again only two
// reductions later, after a barrier that every other CTA reaches only once it
// has read that buffer.  With CL = 1 the cluster steps drop out.
#define TC_CROWS(p) for (int64_t rl = (int64_t)crank * kUpd + threadIdx.x; rl < (p).m; rl += (int64_t)CL * kUpd)

struct ClRed {
    double* post;  // shared [2][kRed]
    int phase;
};

template <int CL> __device__ __forceinline__ void cl_barrier()
{
    if constexpr (CL > 1) cg::this_cluster().sync();
}

// Sums of N doubles over the problem's rows (block_sums_w, then the cluster).
template <int CL, int N> __device__ void cl_sums(double (&v)[N], double (*red)[kRed], ClRed& cr)
{
    block_sums_w<N>(v, red);
    if constexpr (CL > 1) {
        auto cl = cg::this_cluster();
        double* mine = cr.post + cr.phase * kRed;
        if (threadIdx.x < N) mine[threadIdx.x] = red[0][threadIdx.x];  // the CTA's totals
        cl.sync();
        if (threadIdx.x < N) {
            double t = 0.0;
            for (int r = 0; r < CL; ++r) t += cl.map_shared_rank(mine, r)[threadIdx.x];
            red[0][threadIdx.x] = t;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = red[0][i];
        __syncthreads();
        cr.phase ^= 1;
    }
}

// Maximum (take_max) or minimum of a value every thread holds as its CTA's result.
template <int CL> __device__ double cl_fold(double x, bool take_max, ClRed& cr)
{
    if constexpr (CL > 1) {
        auto cl = cg::this_cluster();
        double* mine = cr.post + cr.phase * kRed;
        if (threadIdx.x == 0) mine[0] = x;
        cl.sync();
        x = cl.map_shared_rank(mine, 0)[0];
        for (int r = 1; r < CL; ++r) {
            const double y = cl.map_shared_rank(mine, r)[0];
            x = take_max ? fmax(x, y) : fmin(x, y);
        }
        cr.phase ^= 1;
    }
    return x;
}

// Some thread of the problem's CTAs has flag set.
template <int CL> __device__ bool cl_any(int flag, ClRed& cr)
{
    const int b = __syncthreads_or(flag);
    return cl_fold<CL>(b ? 1.0 : 0.0, true, cr) > 0.0;
}

// Smallest (t, row) over the problem's rows, ties to the lower row.
template <int CL> __device__ void cl_argmin(double& t, int& r, double* sht, int* shr, ClRed& cr)
{
    block_argmin(t, r, sht, shr);
    if constexpr (CL > 1) {
        auto cl = cg::this_cluster();
        double* mine = cr.post + cr.phase * kRed;
        if (threadIdx.x == 0) {
            mine[0] = t;
            mine[1] = (double)r;
        }
        cl.sync();
        for (int q = 0; q < CL; ++q) {
            const double* o = cl.map_shared_rank(mine, q);
            const double t2 = o[0];
            const int r2 = (int)o[1];
            if (t2 < t || (t2 == t && r2 < r)) {
                t = t2;
                r = r2;
            }
        }
        cr.phase ^= 1;
    }
}

// Entries [C0, C0 + NC) of the upper triangle (row-major) of w w^T.
template <int C0, int NC> __device__ __forceinline__ void gram_add(const double (&w)[kBQ], double (&acc)[NC])
{
#pragma unroll
    for (int a = 0; a < kBQ; ++a)
#pragma unroll
        for (int b = a; b < kBQ; ++b) {
            const int e = a * kBQ - a * (a - 1) / 2 + (b - a);
            if (e >= C0 && e < C0 + NC) acc[e - C0] += w[a] * w[b];
        }
}

template <int C0, int NC> __device__ __forceinline__ void gram_store(const double (&acc)[NC], double* A)
{
#pragma unroll
    for (int a = 0; a < kBQ; ++a)
#pragma unroll
        for (int b = a; b < kBQ; ++b) {
            const int e = a * kBQ - a * (a - 1) / 2 + (b - a);
            if (e >= C0 && e < C0 + NC) A[a * kBQ + b] = A[b * kBQ + a] = acc[e - C0];
        }
}

// One chunk of W'^T W' over the variables at a bound in xc whose W' row is not
// zero: the t of a free charge at 0 or pi/2 (a pinned charge's fixed second
// variable has y = s = 0).
template <int CL, int C0, int NC>
__device__ void gram_chunk(const RelaxDev& d, const Prob& p, const int* slot, int hb, double* A, double (*red)[kRed],
                           ClRed& cr, int crank)
{
    double acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.0;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 xc = d.xc[row];
        if (pinned || (lo.x < xc.x && xc.x < hi.x)) continue;
        double wx[kBQ], wy[kBQ];
        w_rows(d, row, slot, hb, wx, wy);
        gram_add<C0, NC>(wx, acc);
    }
    cl_sums<CL, NC>(acc, red, cr);
    if (threadIdx.x == 0) gram_store<C0, NC>(acc, A);
}

template <int CL>
__global__ void __launch_bounds__(kUpd, 1) k_update_lbfgsb(RelaxDev d, const double2* __restrict__ part_g, SlotView v,
                                                         StepParams sp)
{
    __shared__ double sh[kUpd];
    __shared__ int shi[kUpd];
    __shared__ double red[kUpd / 32][kRed];
    __shared__ double aug[kBQ * 2 * kBQ];   // [K | I] -> [I | M]
    __shared__ double Mm[kBQ * kBQ];
    __shared__ double A[kBQ * kBQ];         // W_F^T W_F
    __shared__ double Nv[kBQ * (kBQ + 1)];  // [N | v]
    __shared__ double pv[kBQ], cv[kBQ], mc[kBQ], vv[kBQ], wbs[kBQ], wrs[kBQ];
    __shared__ int slot[kBMem], oth[kBMem];
    __shared__ double bc[4];                // told, dtm, fp, fpp of the Cauchy search
    __shared__ int bflag[2];
    __shared__ double post[2 * kRed];       // this CTA's posts to the cluster's reductions
    __shared__ double bs[kBSmall];          // this CTA's copy of the problem's small products
    const int s = blockIdx.x / CL;
    int crank = 0;
    if constexpr (CL > 1) crank = (int)cg::this_cluster().block_rank();
    const bool lead = crank == 0;          // the CTA that writes the problem's scalars
    ClRed cr{post, 0};
    if (!d.active[s]) return;
    const Prob p = d.prob[s];
    const int k = d.steps[s];
    const int mem = sp.memory;
    const int64_t M = d.M;
    for (int e = threadIdx.x; e < kBSmall; e += kUpd) bs[e] = d.bsmall[(int64_t)s * kBSmall + e];
    __syncthreads();
    double* sy_t = bs;                     // [slot a][slot b] = s_a . y_b
    double* ss_t = sy_t + kBMem * kBMem;   // s_a . s_b
    double* yy_t = ss_t + kBMem * kBMem;   // y_a . y_b
    double* theta_t = yy_t + kBMem * kBMem;  // y.y / s.y of the newest pair

    // 1. dE/d(t, u) of the new point into q, pair statistics, projected-gradient RMS
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // |P(z - g) - z|^2, s.y, s.s, y.y
    bool bad = false;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const double2 g = sum_g(p, rl, part_g, v);
        if (!isfinite(g.x) || !isfinite(g.y)) bad = true;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 z = d.z[row];
        const double2 gz = grad_z(z, g, sp.radius, pinned, true);
        d.q[row] = gz;
        const double px = clampd(z.x - gz.x, lo.x, hi.x) - z.x, py = clampd(z.y - gz.y, lo.y, hi.y) - z.y;
        acc[0] += px * px + py * py;
        if (k > 0) {
            const double2 zo = d.xp[row], go = d.gp[row];
            const double sx = z.x - zo.x, sy = z.y - zo.y, yx = gz.x - go.x, yy = gz.y - go.y;
            acc[1] += sx * yx + sy * yy;
            acc[2] += sx * sx + sy * sy;
            acc[3] += yx * yx + yy * yy;
        }
    }
    if (bad) set_status(d.st, ST_NONFINITE);
    cl_sums<CL, 4>(acc, red, cr);
    const double rms = sqrt(acc[0] / (double)max(p.m, 1));
    if (sp.measure) {
        if (lead && threadIdx.x == 0) d.rms[s] = rms;
        cl_barrier<CL>();  // no CTA leaves while another may still read its posts
        return;
    }
    int hist = d.hist[s], head = d.head[s];
    const bool keep = k > 0 && acc[1] > 1e-12 * sqrt(acc[2]) * sqrt(acc[3]);

    // 2. the kept pair goes to ring slot head; its products with the pairs that stay
    if (keep) {
        if (threadIdx.x == 0) {
            int no = 0;
            for (int a = 0; a < hist; ++a) {
                const int j = ((head - hist + a) % mem + mem) % mem;
                if (j != head) oth[no++] = j;
            }
            for (int a = no; a < kBMem; ++a) oth[a] = -1;
        }
        __syncthreads();
        double dots[4 * (kBMem - 1)];
#pragma unroll
        for (int i = 0; i < 4 * (kBMem - 1); ++i) dots[i] = 0.0;
        TC_CROWS(p)
        {
            const int64_t row = p.row_base + rl;
            const double2 z = d.z[row], zo = d.xp[row], gz = d.q[row], go = d.gp[row];
            const double2 sn = make_double2(z.x - zo.x, z.y - zo.y), yn = make_double2(gz.x - go.x, gz.y - go.y);
#pragma unroll
            for (int o = 0; o < kBMem - 1; ++o) {
                const int j = oth[o];
                if (j < 0) continue;
                const double2 sj = d.Sh[(int64_t)j * M + row], yj = d.Yh[(int64_t)j * M + row];
                dots[4 * o] += sn.x * yj.x + sn.y * yj.y;
                dots[4 * o + 1] += sj.x * yn.x + sj.y * yn.y;
                dots[4 * o + 2] += sn.x * sj.x + sn.y * sj.y;
                dots[4 * o + 3] += yn.x * yj.x + yn.y * yj.y;
            }
            d.Sh[(int64_t)head * M + row] = sn;
            d.Yh[(int64_t)head * M + row] = yn;
            d.gp[row] = gz;
        }
        cl_sums<CL, 4 * (kBMem - 1)>(dots, red, cr);
        if (threadIdx.x == 0) {
            for (int o = 0; o < kBMem - 1; ++o) {
                const int j = oth[o];
                if (j < 0) continue;
                sy_t[head * kBMem + j] = dots[4 * o];
                sy_t[j * kBMem + head] = dots[4 * o + 1];
                ss_t[head * kBMem + j] = ss_t[j * kBMem + head] = dots[4 * o + 2];
                yy_t[head * kBMem + j] = yy_t[j * kBMem + head] = dots[4 * o + 3];
            }
            sy_t[head * kBMem + head] = acc[1];
            ss_t[head * kBMem + head] = acc[2];
            yy_t[head * kBMem + head] = acc[3];
            *theta_t = acc[3] / acc[1];
        }
        __syncthreads();
        if (lead)
            for (int e = threadIdx.x; e < kBSmall; e += kUpd) d.bsmall[(int64_t)s * kBSmall + e] = bs[e];
        head = (head + 1) % mem;
        hist = min(hist + 1, mem);
    } else {
        TC_CROWS(p) d.gp[p.row_base + rl] = d.q[p.row_base + rl];
    }
    if (sp.gtol > 0.0 && rms < sp.gtol) {
        if (lead && threadIdx.x == 0) {
            d.active[s] = 0;
            d.rms[s] = rms;
            d.hist[s] = hist;
            d.head[s] = head;
        }
        cl_barrier<CL>();
        return;
    }
    __syncthreads();

    // 3. M = K^{-1}
    const int hb = hist;
    const double theta = hb > 0 ? *theta_t : 1.0 / sp.step0;
    if (threadIdx.x < kBMem) slot[threadIdx.x] = threadIdx.x < hb ? ((head - hb + (int)threadIdx.x) % mem + mem) % mem : 0;
    __syncthreads();
    for (int e = threadIdx.x; e < kBQ * kBQ; e += kUpd) {
        const int a = e / kBQ, b = e % kBQ;
        const bool ya = a < kBMem, yb = b < kBMem;
        const int ia = ya ? a : a - kBMem, ib = yb ? b : b - kBMem;
        double val;
        if (ia >= hb || ib >= hb) {
            val = a == b ? 1.0 : 0.0;
        } else {
            const int ja = slot[ia], jb = slot[ib];
            if (ya && yb)
                val = ia == ib ? -sy_t[ja * kBMem + ja] : 0.0;  // -D
            else if (ya)
                val = ib > ia ? sy_t[jb * kBMem + ja] : 0.0;    // L^T: s_ib . y_ia
            else if (yb)
                val = ia > ib ? sy_t[ja * kBMem + jb] : 0.0;    // L: s_ia . y_ib
            else
                val = theta * ss_t[ja * kBMem + jb];            // theta S S^T
        }
        aug[a * 2 * kBQ + b] = val;
        aug[a * 2 * kBQ + kBQ + b] = a == b ? 1.0 : 0.0;
    }
    __syncthreads();
    {
        const bool ok = block_gauss_jordan(aug, pv, shi);  // pv, shi: scratch until the Cauchy search
        if (threadIdx.x == 0) bflag[0] = ok ? 1 : 0;
    }
    __syncthreads();
    if (!bflag[0]) {
        set_status(d.st, ST_NONFINITE);
        if (lead && threadIdx.x == 0) d.active[s] = 0;
        cl_barrier<CL>();
        return;
    }
    for (int e = threadIdx.x; e < kBQ * kBQ; e += kUpd) Mm[e] = aug[(e / kBQ) * 2 * kBQ + kBQ + e % kBQ];

    // 4. generalized Cauchy point: d = -g except where the breakpoint is 0,
    //    p = W^T d, breakpoints of the t variables
    double pd[kBQ + 1];
#pragma unroll
    for (int i = 0; i <= kBQ; ++i) pd[i] = 0.0;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 z = d.z[row], gz = d.gp[row];
        const double tx = breakpoint(z.x, gz.x, lo.x, hi.x), ty = breakpoint(z.y, gz.y, lo.y, hi.y);
        const double2 dv = make_double2(tx == 0.0 ? 0.0 : -gz.x, ty == 0.0 ? 0.0 : -gz.y);
        d.q[row] = dv;
        d.bp[row] = tx > 0.0 && tx < INFINITY ? tx : INFINITY;  // only a t variable has a finite one
        double wx[kBQ], wy[kBQ];
        w_rows(d, row, slot, hb, wx, wy);
#pragma unroll
        for (int a = 0; a < kBQ; ++a) pd[a] += wx[a] * dv.x + wy[a] * dv.y;
        pd[kBQ] += dv.x * dv.x + dv.y * dv.y;
    }
    cl_sums<CL, kBQ + 1>(pd, red, cr);
    // The small dense algebra runs on warp 0, one lane per entry: a float64
    // instruction of one thread takes the SM's float64 pipe as long as a warp's.
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        if (lane == 0)
            for (int a = 0; a < kBQ; ++a) {
                pv[a] = a < kBMem ? pd[a] : theta * pd[a];  // p = D W'^T d
                cv[a] = 0.0;
            }
        __syncwarp();
        const double mp = lane < kBQ ? row_dot16(Mm, pv, lane) : 0.0;
        const double pmp = lanes_sum16(lane < kBQ ? pv[lane] * mp : 0.0);
        if (lane == 0) {
            const double fp = -pd[kBQ];
            const double fpp = -theta * fp - pmp;
            bc[0] = 0.0;
            bc[1] = fpp > 0.0 ? -fp / fpp : 0.0;
            bc[2] = fp;
            bc[3] = fpp;
            bflag[1] = fpp > 0.0 ? 1 : 0;
        }
    }
    __syncthreads();
    const double fpp0 = bc[3];
    const bool moves = fpp0 > 0.0;
    // visit the breakpoints in increasing (t, row) while the segment minimiser lies beyond them;
    // each thread keeps the smallest (t, row) of its own rows and rescans them only when the
    // breakpoint just fixed was one of them
    double own_t = INFINITY;
    int own_r = INT_MAX;
    TC_CROWS(p)
    {
        const double t = d.bp[p.row_base + rl];
        if (t > 0.0 && t < own_t) {
            own_t = t;
            own_r = (int)rl;
        }
    }
    while (bflag[1]) {
        double tmin = own_t;
        int rmin = own_r;
        cl_argmin<CL>(tmin, rmin, sh, shi, cr);
        // every CTA holds the same (tmin, rmin) and bc, so all take the same branch
        const double told = bc[0], dtm = bc[1];
        const double dt = tmin - told;
        if (rmin == INT_MAX || dtm < dt) {
            __syncthreads();
            if (threadIdx.x == 0) bflag[1] = 0;
            __syncthreads();
            break;
        }
        const int64_t b = p.row_base + rmin;
        const int orank = (rmin / kUpd) % CL;  // the CTA that holds row b
        // the row's own CTA posts what the search needs of row b: g, the bound it reaches, z, and
        // its row of W' (unscaled); the others read the post after the cluster barrier
        double* bpost = cr.post + cr.phase * kRed;
        if (orank == crank && threadIdx.x < 32) {
            if (lane == 0) {
                const bool pinned = d.flags && d.flags[d.gidx[b]];
                double2 lo, hi;
                tu_bounds(pinned, lo, hi);
                bpost[0] = d.gp[b].x;
                bpost[1] = d.q[b].x > 0.0 ? hi.x : lo.x;
                bpost[2] = d.z[b].x;
            }
            if (lane < kBQ) {
                const int ia = lane < kBMem ? lane : lane - kBMem;
                double w = 0.0;
                if (ia < hb) {
                    const int64_t o = (int64_t)slot[ia] * M + b;
                    w = lane < kBMem ? d.Yh[o].x : d.Sh[o].x;
                }
                bpost[3 + lane] = w;
            }
        }
        if constexpr (CL > 1) cg::this_cluster().sync(); else __syncthreads();
        const double* opost = bpost;
        if constexpr (CL > 1) opost = cg::this_cluster().map_shared_rank(bpost, orank);
        if (threadIdx.x < 32) {
            const double gb = opost[0], xb = opost[1], zb = xb - opost[2];
            double wa = 0.0;  // entry `lane` of w_b (row b of W, variable t)
            if (lane < kBQ) {
                wa = lane < kBMem ? opost[3 + lane] : theta * opost[3 + lane];
                wbs[lane] = wa;
                cv[lane] += dt * pv[lane];
            }
            __syncwarp();
            double mcl = 0.0, mpl = 0.0, mwl = 0.0;
            if (lane < kBQ) {
                mcl = row_dot16(Mm, cv, lane);
                mpl = row_dot16(Mm, pv, lane);
                mwl = row_dot16(Mm, wbs, lane);
            }
            const double wMc = lanes_sum16(wa * mcl), wMp = lanes_sum16(wa * mpl), wMw = lanes_sum16(wa * mwl);
            __syncwarp();
            if (lane < kBQ) pv[lane] += gb * wa;
            if (lane == 0) {
                double fp = bc[2], fpp = bc[3];
                fp = __dsub_rn(__dadd_rn(__dadd_rn(__dadd_rn(fp, __dmul_rn(dt, fpp)), __dmul_rn(gb, gb)),
                                         __dmul_rn(__dmul_rn(theta, gb), zb)),
                               __dmul_rn(gb, wMc));
                fpp = __dsub_rn(__dsub_rn(__dsub_rn(fpp, __dmul_rn(__dmul_rn(theta, gb), gb)),
                                          __dmul_rn(__dmul_rn(2.0, gb), wMp)),
                                __dmul_rn(__dmul_rn(gb, gb), wMw));
                if (fpp < 0x1p-52 * fpp0) fpp = 0x1p-52 * fpp0;
                if (orank == crank) {  // only the row's own CTA writes it
                    d.bp[b] = -1.0;    // fixed at its bound
                    reinterpret_cast<double*>(d.xc + b)[0] = xb;
                }
                bc[0] = tmin;
                bc[1] = -fp / fpp;
                bc[2] = fp;
                bc[3] = fpp;
            }
        }
        cr.phase ^= 1;
        __syncthreads();
        if (orank == crank) {
            // the owner's warp rescans the owner's rows, 32 at a time
            const int owner = rmin % kUpd;
            if ((int)(threadIdx.x >> 5) == (owner >> 5)) {
                double tb = INFINITY;
                int rb_ = INT_MAX;
                for (int64_t rl = owner + (int64_t)kUpd * (crank + (int64_t)CL * lane); rl < p.m;
                     rl += 32LL * CL * kUpd) {
                    const double t = d.bp[p.row_base + rl];
                    if (t > 0.0 && t < tb) {
                        tb = t;
                        rb_ = (int)rl;
                    }
                }
                warp_argmin(tb, rb_);
                if ((int)threadIdx.x == owner) {
                    own_t = tb;
                    own_r = rb_;
                }
            }
        }
    }
    if (threadIdx.x < 32 && moves) {
        const double dtm = fmax(bc[1], 0.0);
        if (lane < kBQ) cv[lane] += dtm * pv[lane];
        __syncwarp();
        if (lane == 0) bc[0] += dtm;
    }
    __syncthreads();
    {
        const double told = bc[0];
        TC_CROWS(p)
        {
            const int64_t row = p.row_base + rl;
            const double2 z = d.z[row], dv = d.q[row];
            const double xcx = d.bp[row] == -1.0 ? d.xc[row].x : (moves ? z.x + told * dv.x : z.x);
            d.xc[row] = make_double2(xcx, moves ? z.y + told * dv.y : z.y);
        }
    }

    // 5. subspace minimisation over the free variables (direct primal method)
    if (threadIdx.x < kBQ) {
        const double t = row_dot16(Mm, cv, threadIdx.x);
        mc[threadIdx.x] = threadIdx.x < kBMem ? t : theta * t;  // D M c: a row of W' dotted with it is w . M c
    }
    __syncthreads();
    double wr[kBQ];
#pragma unroll
    for (int a = 0; a < kBQ; ++a) wr[a] = 0.0;
    int bound_rows = 0;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 z = d.z[row], gz = d.gp[row], xc = d.xc[row];
        double wx[kBQ], wy[kBQ];
        w_rows(d, row, slot, hb, wx, wy);
        const bool fx = lo.x < xc.x && xc.x < hi.x, fy = lo.y < xc.y && xc.y < hi.y;
        if (!pinned && !fx) bound_rows = 1;
        const double rx = fx ? gz.x + theta * (xc.x - z.x) - dot16(wx, mc) : 0.0;
        const double ry = fy ? gz.y + theta * (xc.y - z.y) - dot16(wy, mc) : 0.0;
        d.q[row] = make_double2(rx, ry);
#pragma unroll
        for (int a = 0; a < kBQ; ++a) wr[a] += wx[a] * rx + wy[a] * ry;
    }
    cl_sums<CL, kBQ>(wr, red, cr);
    // W'^T W' over every variable, from the kept products (into aug, free after the inversion)
    for (int e = threadIdx.x; e < kBQ * kBQ; e += kUpd) {
        const int a = e / kBQ, b = e % kBQ;
        const bool ya = a < kBMem, yb = b < kBMem;
        const int ia = ya ? a : a - kBMem, ib = yb ? b : b - kBMem;
        double val = 0.0;
        if (ia < hb && ib < hb) {
            const int ja = slot[ia], jb = slot[ib];
            if (ya && yb)
                val = yy_t[ja * kBMem + jb];
            else if (ya)
                val = sy_t[jb * kBMem + ja];  // y_ia . s_ib
            else if (yb)
                val = sy_t[ja * kBMem + jb];  // s_ia . y_ib
            else
                val = ss_t[ja * kBMem + jb];
        }
        aug[e] = val;
    }
    // less the rows at a bound
    if (cl_any<CL>(bound_rows, cr)) {
        gram_chunk<CL, 0, 34>(d, p, slot, hb, A, red, cr, crank);
        gram_chunk<CL, 34, 34>(d, p, slot, hb, A, red, cr, crank);
        gram_chunk<CL, 68, 34>(d, p, slot, hb, A, red, cr, crank);
        gram_chunk<CL, 102, 34>(d, p, slot, hb, A, red, cr, crank);
    } else if (threadIdx.x == 0) {
        for (int e = 0; e < kBQ * kBQ; ++e) A[e] = 0.0;
    }
    __syncthreads();
    static_assert(kBQ * kBQ == kUpd, "one entry of the small matrices per thread");
    constexpr int ld = kBQ + 1;
    {
        // W_F^T W_F = D (W'^T W' - bound rows) D and W_F^T r = D W'^T r
        const int e = threadIdx.x;
        const double sa = e / kBQ < kBMem ? 1.0 : theta, sb = e % kBQ < kBMem ? 1.0 : theta;
        A[e] = (aug[e] - A[e]) * sa * sb;
        if (e < kBQ) {
            double w = 0.0;
#pragma unroll
            for (int i = 0; i < kBQ; ++i)
                if (i == e) w = wr[i];
            wrs[e] = e < kBMem ? w : theta * w;
        }
    }
    __syncthreads();
    {
        // N = I - M A / theta (one entry per thread) and its right-hand side M D W'^T r
        const int e = threadIdx.x, ea = e / kBQ, eb = e % kBQ;
        double t = 0.0;
        for (int q = 0; q < kBQ; ++q) t += Mm[ea * kBQ + q] * A[q * kBQ + eb];
        Nv[ea * ld + eb] = __dsub_rn(ea == eb ? 1.0 : 0.0, __ddiv_rn(t, theta));
        if (e < kBQ) Nv[e * ld + kBQ] = row_dot16(Mm, wrs, e);
    }
    __syncthreads();
    // Gauss elimination with partial pivoting on [N | v], the whole CTA taking part; every entry
    // sees the same operations in the same order as a one-lane-per-column elimination
    // per column, warp 0 finds the pivot, swaps the rows and forms the multipliers (one CTA
    // barrier), then the CTA eliminates (a second barrier)
    bool ok = true;
    for (int col = 0; col < kBQ; ++col) {
        if (threadIdx.x < 32) {
            const int piv = warp_pivot(Nv, ld, col);
            if (threadIdx.x == 0) shi[0] = piv;
            if (piv >= 0) {
                if (piv != col) {
                    double a = 0.0, b = 0.0;
                    if (threadIdx.x <= kBQ) {
                        a = Nv[col * ld + threadIdx.x];
                        b = Nv[piv * ld + threadIdx.x];
                    }
                    __syncwarp();
                    if (threadIdx.x <= kBQ) {
                        Nv[col * ld + threadIdx.x] = b;
                        Nv[piv * ld + threadIdx.x] = a;
                    }
                    __syncwarp();
                }
                if ((int)threadIdx.x > col && threadIdx.x < kBQ)
                    pv[threadIdx.x] = __ddiv_rn(Nv[threadIdx.x * ld + col], Nv[col * ld + col]);
            }
        }
        __syncthreads();
        if (shi[0] < 0) {
            ok = false;
            break;
        }
        for (int e = threadIdx.x; e < kBQ * ld; e += kUpd) {
            const int r = e / ld, c = e % ld;
            if (r > col && c >= col) Nv[e] = __dsub_rn(Nv[e], __dmul_rn(pv[r], Nv[col * ld + c]));
        }
        __syncthreads();
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (ok)
            for (int a = kBQ - 1; a >= 0; --a) {
                // v_a = (rhs_a - sum_{q > a} N_aq v_q) / N_aa, the products on lanes a+1 .. kBQ-1
                const double t = lanes_sum16(lane > a && lane < kBQ ? __dmul_rn(Nv[a * ld + lane], vv[lane]) : 0.0);
                if (lane == 0) vv[a] = __ddiv_rn(__dsub_rn(Nv[a * ld + kBQ], t), Nv[a * ld + a]);
                __syncwarp();
            }
        if (lane >= kBMem && lane < kBQ) vv[lane] *= theta;  // D v: a row of W' dotted with it is w . v
        if (lane == 0) bflag[0] = ok ? 1 : 0;
    }
    __syncthreads();
    if (!bflag[0]) {
        set_status(d.st, ST_NONFINITE);
        if (lead && threadIdx.x == 0) d.active[s] = 0;
        cl_barrier<CL>();
        return;
    }
    double amin = 1.0;
    const double ith = 1.0 / theta, ith2 = ith * ith;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 r = d.q[row], xc = d.xc[row];
        double wx[kBQ], wy[kBQ];
        w_rows(d, row, slot, hb, wx, wy);
        const bool fx = lo.x < xc.x && xc.x < hi.x, fy = lo.y < xc.y && xc.y < hi.y;
        const double dux = fx ? -r.x * ith - dot16(wx, vv) * ith2 : 0.0;
        const double duy = fy ? -r.y * ith - dot16(wy, vv) * ith2 : 0.0;
        if (fx && dux > 0.0 && hi.x < INFINITY) amin = fmin(amin, (hi.x - xc.x) / dux);
        if (fx && dux < 0.0 && lo.x > -INFINITY) amin = fmin(amin, (lo.x - xc.x) / dux);
        if (fy && duy > 0.0 && hi.y < INFINITY) amin = fmin(amin, (hi.y - xc.y) / duy);
        if (fy && duy < 0.0 && lo.y > -INFINITY) amin = fmin(amin, (lo.y - xc.y) / duy);
        d.q[row] = make_double2(dux, duy);
    }
    sh[threadIdx.x] = amin;
    __syncthreads();
    for (int w = kUpd / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    double astar = sh[0];
    __syncthreads();
    astar = cl_fold<CL>(astar, false, cr);

    // 6. direction xbar - z, descent check, capped step
    double gd[1] = {0.0};
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 z = d.z[row], gz = d.gp[row], xc = d.xc[row], du = d.q[row];
        const double bx = lo.x < xc.x && xc.x < hi.x ? xc.x + astar * du.x : xc.x;
        const double by = lo.y < xc.y && xc.y < hi.y ? xc.y + astar * du.y : xc.y;
        const double2 dv = make_double2(bx - z.x, by - z.y);
        d.q[row] = dv;
        gd[0] += gz.x * dv.x + gz.y * dv.y;
    }
    cl_sums<CL, 1>(gd, red, cr);
    const bool reset = gd[0] >= 0.0;
    if (reset) {
        hist = 0;
        head = 0;
    }
    double dmax = 0.0;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        double2 dv = d.q[row];
        if (reset) {
            const bool pinned = d.flags && d.flags[d.gidx[row]];
            double2 lo, hi;
            tu_bounds(pinned, lo, hi);
            const double2 z = d.z[row], gz = d.gp[row];
            dv = make_double2(clampd(z.x - sp.step0 * gz.x, lo.x, hi.x) - z.x,
                              clampd(z.y - sp.step0 * gz.y, lo.y, hi.y) - z.y);
            d.q[row] = dv;
        }
        dmax = fmax(dmax, sqrt(dv.x * dv.x + dv.y * dv.y));
    }
    dmax = cl_fold<CL>(block_max(dmax, sh), true, cr);
    const double alpha = dmax > sp.maxstep ? sp.maxstep / dmax : 1.0;
    if (lead && threadIdx.x == 0 && d.ls_alpha) d.ls_alpha[s] = alpha;
    TC_CROWS(p)
    {
        const int64_t row = p.row_base + rl;
        const bool pinned = d.flags && d.flags[d.gidx[row]];
        double2 lo, hi;
        tu_bounds(pinned, lo, hi);
        const double2 z = d.z[row], dv = d.q[row];
        d.xp[row] = z;
        if (d.xold) d.xold[row] = d.x[row];
        const double2 zn = make_double2(clampd(z.x + alpha * dv.x, lo.x, hi.x), clampd(z.y + alpha * dv.y, lo.y, hi.y));
        d.z[row] = zn;
        const double2 xn = z_to_x(zn, sp.radius, pinned, true);
        d.x[row] = xn;
        d.xs[row] = split4(xn.x, xn.y);
        if (d.x3) d.x3[row] = split3(xn.x, xn.y);
    }
    if (lead && threadIdx.x == 0) {
        d.steps[s] = k + 1;
        d.rms[s] = rms;
        d.hist[s] = hist;
        d.head[s] = head;
    }
    cl_barrier<CL>();
}
