// tc_device.cuh -- device arithmetic and the generic pair pass of libtc.
//
// Everything the kernels compute is a sum over (target row, source charge)
// pairs of the 1/r Coulomb interaction of Eq. (hamiltonian):
//     e-term  1/|r_i - r_j|,   gradient term  -(r_i - r_j)/|r_i - r_j|^3,
// or, for the pairwise energy change of Sec. II D, the difference of two such
// e-terms.  Rows are the moving charges of a problem; sources are tiles of
// either the fixed configuration (the "snapshot", with the problem's own
// charges masked out) or the problem's own moving charges.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

// Device status codes (same numbering as tc_status).
enum : int { ST_OK = 0, ST_INVALID = 1, ST_NONFINITE = 3, ST_OUTSIDE = 4, ST_TIMEOUT = 5 };

// A masked-out or padding source sits this far away: its 1/r term is below
// 1e-18 and its gradient term below 1e-36, so even 255 of them change no real
// row sum by more than a rounding.  Every squared distance to such a source
// (< 1e37) stays inside the float32 range the rsqrt seed of rsqrt64 needs.
constexpr double kFar64 = 1.0e18;
constexpr float kFar32 = 1.0e18f;
// Rows past the end of a problem sit at the opposite far corner, so they
// never coincide with a far source.
constexpr double kFarRow64 = -1.0e18;
constexpr float kFarRow32 = -1.0e18f;

// Slack above the wall radius that still counts as inside (Eq. potential).
constexpr double kWallSlack = 1e-12;

__device__ __forceinline__ void set_status(int* st, int code)
{
    if (st) atomicCAS(st, 0, code);
}

// One MUFU.RSQ: approximate 1/sqrt(x) in float32 (denormal inputs flush to 0).
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One MUFU.RCP: approximate 1/x in float32.
__device__ __forceinline__ float rcp_mufu(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// float64 1/sqrt(r2): a float32 seed y0, then one correction step of the
// binomial series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3) with
// e = 1 - r2 y0^2.
//
// The seed avoids float64<->float32 conversion instructions, which occupy the
// (on B300 very narrow) float64 pipe: the high word of r2 holds its sign, 11
// exponent bits and top 20 mantissa bits, and rebiasing the exponent
// (1023 -> 127, i.e. subtracting 896 << 20) and shifting left by 3 gives the
// float32 with r2's mantissa truncated to 20 bits (relative error < 2^-20);
// MUFU.RSQ of it, widened back exactly (exponent +896, mantissa bits moved
// down by 3 into the high word and 29 into the low word), has |e| < 2^-19, so
// the cubic remainder (5/16) e^3 stays below 2^-58 relative and the result is
// within a few roundings of the correctly rounded value.  Integer work runs on
// the ALU pipe.  Valid for 2^-126 <= r2 < 2^128; r2 below that (coincident
// charges) gives NaN, which the finiteness checks report.
__device__ __forceinline__ double rsqrt64(double r2)
{
    const unsigned hi = (unsigned)__double2hiint(r2);
    const float seed = __uint_as_float((hi - (896u << 20)) << 3);
    const unsigned fb = __float_as_uint(rsqrt_mufu(seed));
    double y0 = __hiloint2double((int)((fb >> 3) + (896u << 20)), (int)(fb << 29));
    // r2 below 2^-126 (coincident charges) has no float seed: make the result NaN
    y0 = hi < (897u << 20) ? __longlong_as_double(0x7ff8000000000000LL) : y0;
    const double t = r2 * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(0.375, e, 0.5);
    const double q = e * p;
    return fma(y0, q, y0);
}

// Error-free transformation of a float32 sum (Knuth's TwoSum): hi + v is
// split into its rounded value and the exact rounding error, which is kept in
// lo.  Used to carry float32 tile sums across tiles without float64 work.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v)
{
    float s = hi + v;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

// Same transformation in float64, used for the energy row sums.
__device__ __forceinline__ void dd_add(double& hi, double& lo, double v)
{
    double s = hi + v;
    double bp = s - hi;
    double err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

// hi/lo split of a float64 coordinate: hi = rn(x), lo = rn(x - hi).
__device__ __forceinline__ float4 split4(double x, double y)
{
    float xh = (float)x, yh = (float)y;
    return make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
}

// ------------------------------------------------------------ stream-K ---
// The pass work is a list of W equal units (one row block x one source tile),
// cut into G contiguous ranges [b_k, b_{k+1}), b_k = floor(W k / G), one per
// persistent CTA (the stream-K decomposition of Osama et al., PPoPP 2023).
// owner(u) is the CTA whose range holds unit u: the largest k with
// floor(W k / G) <= u, i.e. k = ceil(G (u + 1) / W) - 1.
__host__ __device__ __forceinline__ int64_t sk_begin(int64_t W, int64_t G, int64_t k)
{
    return (W * k) / G;
}

__host__ __device__ __forceinline__ int64_t sk_owner(int64_t u, int64_t W, int64_t G)
{
    return (G * (u + 1) + W - 1) / W - 1;
}

// One problem of a pass: rows [row_base, row_base + m) of the row arrays move;
// sources are the snapshot range [snap_b, snap_e) of the configuration (with
// the problem's own charges masked by mask words [mask_off, ...)) followed by
// the problem's own rows.
struct Prob {
    int64_t row_base;
    int64_t snap_b, snap_e;
    int64_t unit_off;   // first pass unit of this problem
    int64_t mask_off;   // first mask word, -1 without a mask
    int32_t m;          // rows
    int32_t n_rb;       // row blocks
    int32_t n_t_snap;   // snapshot tiles
    int32_t n_t_priv;   // own-row tiles
};

__device__ __forceinline__ int find_prob(const Prob* __restrict__ P, int S, int64_t u)
{
    // largest s with P[s].unit_off <= u (problems are ordered by unit_off)
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P[mid].unit_off <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// (x_old, y_old, x_new, y_new) of one moving charge, 32-byte aligned.
struct alignas(32) d4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ d4 make_d4(double x, double y, double z, double w)
{
    d4 r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.w = w;
    return r;
}

// A charge for the difference-form energy change: old position split hi/lo
// and its move new - old in float32 (zero for charges that stay), 32 bytes.
struct alignas(32) f8 {
    float4 p;   // (x_hi, y_hi, x_lo, y_lo) of the old position
    float2 d;   // move (dx, dy)
    float2 pad;
};
__host__ __device__ __forceinline__ f8 make_f8(float4 p, float dx, float dy)
{
    f8 r;
    r.p = p;
    r.d = make_float2(dx, dy);
    r.pad = make_float2(0.f, 0.f);
    return r;
}

// A coordinate pair split into three float32 parts for the float64-grade
// float32 pass: x = hi + mid + lo with hi on the grid 2^-21, mid on the grid
// 2^-44 and lo the float32 rounding of the rest (|lo| <= 2^-45, error <= 2^-69).
// For |x| <= 1 the differences of two his and of two mids are exact in
// float32 (at most 23 and 24 significant bits), so a separation is known to
// ~2^-69 before any arithmetic.  Values beyond the disk (far sentinels) keep
// hi = (float)x and zero mid and lo.
struct alignas(32) fx3 {
    float4 hm;  // (x_hi, y_hi, x_mid, y_mid)
    float2 lo;  // (x_lo, y_lo)
    float2 pad;
};

__host__ __device__ __forceinline__ void split3_1(double x, float& h, float& m, float& l)
{
    if (!(fabs(x) <= 2.0)) {
        h = (float)x;
        m = 0.f;
        l = 0.f;
        return;
    }
    const double hd = rint(x * 2097152.0) * (1.0 / 2097152.0);   // 2^21
    const double r1 = x - hd;                                      // exact, |r1| <= 2^-22
    const double md = rint(r1 * 17592186044416.0) * (1.0 / 17592186044416.0);  // 2^44
    h = (float)hd;
    m = (float)md;
    l = (float)(r1 - md);
}

__host__ __device__ __forceinline__ fx3 split3(double x, double y)
{
    fx3 r;
    float xh, xm, xl, yh, ym, yl;
    split3_1(x, xh, xm, xl);
    split3_1(y, yh, ym, yl);
    r.hm = make_float4(xh, yh, xm, ym);
    r.lo = make_float2(xl, yl);
    r.pad = make_float2(0.f, 0.f);
    return r;
}

__host__ __device__ __forceinline__ fx3 far3(float v)
{
    fx3 r;
    r.hm = make_float4(v, v, 0.f, 0.f);
    r.lo = make_float2(0.f, 0.f);
    r.pad = make_float2(0.f, 0.f);
    return r;
}

// Pass flavours.
enum PassKind { PASS_MIXED = 0, PASS_F64 = 1, PASS_DELTA = 2, PASS_DMIX = 3, PASS_F64X = 4 };

template <int KIND> struct SrcT;
template <> struct SrcT<PASS_MIXED> { using type = float4; };   // (x_hi, y_hi, x_lo, y_lo)
template <> struct SrcT<PASS_F64> { using type = double2; };    // (x, y)
template <> struct SrcT<PASS_DELTA> { using type = d4; };  // (x_old, y_old, x_new, y_new)
template <> struct SrcT<PASS_DMIX> { using type = f8; };   // old split + move
template <> struct SrcT<PASS_F64X> { using type = fx3; };  // three-part split

// Arguments of one pass launch.
struct PassArgs {
    const Prob* prob;   // device table of S problems; nullptr: the single problem below
    Prob single;
    int S;              // problems
    int64_t W;          // total units
    int64_t M;          // total rows (row arrays and partial-slot stride)
    const void* rows;   // row positions: float4 split (mixed), double2 (f64), d4 old/new (delta),
                        // f8 old split + move (difference form)
    const void* snap;   // snapshot: float4 split (mixed, difference form), double2 (f64, delta)
    const uint32_t* mask;
    const int* active;  // nullable; problems with active[s] == 0 are skipped
    double* part_e;     // [slots x M] row partial energies (or energy changes)
    double2* part_g;    // [slots x M] row partial gradients (nullable)
    // nullable: the launch's G ranges are taken in order from this ticket counter (zero between
    // launches) by `ctas` persistent CTAs instead of one range per CTA; `ranges` is set to G at
    // the launch
    unsigned* ticket;
    int64_t ctas;
    int64_t ranges;
    // float64 pass, problems without snapshot tiles (all pairs of a world): 1 = each unordered pair
    // once.  Row block rb covers the problem's own tiles 2 rb and 2 rb + 1; units of earlier tiles
    // do nothing, those two tiles are computed as usual (every ordered pair, rows only), and a
    // later tile t adds each pair's terms to the row and to the source: the source sums of unit
    // (rb, t) go to col_e / col_g[rb * col_stride + row - row_sub] for the rows of tile t.
    int sym;
    double* col_e;
    double2* col_g;
    int64_t col_stride;
};

}  // namespace tc
