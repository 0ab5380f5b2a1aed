// tc_order.cu -- structure analysis of Sec. III: Voronoi neighbours, coordination
// numbers and the sixfold bond-orientational order of Eq. (psi6).
//
// One thread per charge builds its Voronoi cell by clipping a square with the
// perpendicular bisector of every other charge that can still cut it, in
// float64, labelling each cell edge with the charge whose bisector made it.
// The square is large (1e6) because the Voronoi edge of a convex-hull edge is
// a ray that can start far outside the disk (at the circumcentre of a thin
// triangle along the hull).
// The charges whose labels survive are the Voronoi neighbours.  A charge p can
// only cut the cell if |p - r_i| < 2 R, R the largest distance from r_i to a
// vertex of the current cell; every thread scans all n charges from shared
// memory in float32 with a safety margin on that test, after first clipping
// with its 16 nearest charges (found by a first scan), which makes R small.
#include <algorithm>

#include "tc_plan.cuh"

namespace tc {

namespace {

constexpr int kOrdThreads = 128;
constexpr int kMaxPoly = 40;   // vertices of a cell while clipping
constexpr int kNear = 16;      // nearest charges clipped first
constexpr double kBox = 1.0e6; // initial cell: the square [-1e6, 1e6]^2 (the disk is [-1, 1]^2)
constexpr int kZBins = 16;     // P(z) bins; the last holds z >= 15

struct Poly {
    double x[kMaxPoly], y[kMaxPoly];
    int lab[kMaxPoly];  // edge k runs from vertex k to vertex k+1 and lies on lab[k]'s bisector
    int nv;
};

// Clip `a` (the cell of r) by the half-plane nearer to r than to q (label j);
// the result goes to `b`.  Returns false (no change, b untouched) when no
// vertex lies strictly on q's side; sets *overflow when kMaxPoly is exceeded.
__device__ bool clip(const Poly& a, Poly& b, double2 r, double2 q, int j, bool* overflow)
{
    const double dx = q.x - r.x, dy = q.y - r.y;
    const double mx = 0.5 * (q.x + r.x), my = 0.5 * (q.y + r.y);
    double s[kMaxPoly];
    bool cut = false;
    for (int k = 0; k < a.nv; ++k) {
        s[k] = (a.x[k] - mx) * dx + (a.y[k] - my) * dy;
        cut |= s[k] > 0.0;
    }
    if (!cut) return false;
    int m = 0;
    for (int k = 0; k < a.nv; ++k) {
        const int k1 = k + 1 == a.nv ? 0 : k + 1;
        const bool in0 = s[k] <= 0.0, in1 = s[k1] <= 0.0;
        if (in0) {
            if (m >= kMaxPoly) { *overflow = true; return false; }
            b.x[m] = a.x[k]; b.y[m] = a.y[k]; b.lab[m] = a.lab[k]; ++m;
        }
        if (in0 != in1) {
            const double t = s[k] / (s[k] - s[k1]);
            if (m >= kMaxPoly) { *overflow = true; return false; }
            b.x[m] = a.x[k] + t * (a.x[k1] - a.x[k]);
            b.y[m] = a.y[k] + t * (a.y[k1] - a.y[k]);
            // leaving the half-plane: the new edge lies on j's bisector; entering: the old edge goes on
            b.lab[m] = in0 ? j : a.lab[k];
            ++m;
        }
    }
    b.nv = m;
    return true;
}

__device__ double far2(const Poly& a, double2 r)
{
    double m = 0.0;
    for (int k = 0; k < a.nv; ++k) {
        const double dx = a.x[k] - r.x, dy = a.y[k] - r.y;
        m = fmax(m, dx * dx + dy * dy);
    }
    return m;
}

// Float32 reject threshold: a charge whose float32 squared distance is at least
// this cannot cut the cell (|p - r| >= 2R; float32 positions and arithmetic
// move a distance of at most ~2e-7 and a square by a relative 3e-7).
__device__ float reject_limit(double R2)
{
    const double R = sqrt(R2);
    const double lim = (2.0 * R + 2.5e-7) * (2.0 * R + 2.5e-7) * (1.0 + 1e-6);
    return lim > 3.0e38 ? 3.0e38f : (float)lim;
}

__global__ void k_to_float2(const double2* __restrict__ pos, int64_t n, float2* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)pos[i].x, (float)pos[i].y);
}

__global__ void __launch_bounds__(kOrdThreads) k_voronoi(const double2* __restrict__ pos,
                                                         const float2* __restrict__ posf, int64_t n,
                                                         int32_t* __restrict__ z, double2* __restrict__ psi,
                                                         int32_t* __restrict__ nbr, int max_nbr, int* st)
{
    __shared__ float2 tile[kOrdThreads];
    const int tid = threadIdx.x;
    const int64_t i = blockIdx.x * (int64_t)kOrdThreads + tid;
    const bool act = i < n;
    Poly A, B;
    Poly* cur = &A;
    Poly* nxt = &B;
    bool overflow = false, coincident = false;
    const double2 r = act ? pos[i] : make_double2(0.0, 0.0);
    const float2 rf = make_float2((float)r.x, (float)r.y);
    A.nv = 4;
    A.x[0] = -kBox; A.y[0] = -kBox; A.lab[0] = -1;
    A.x[1] = kBox;  A.y[1] = -kBox; A.lab[1] = -1;
    A.x[2] = kBox;  A.y[2] = kBox;  A.lab[2] = -1;
    A.x[3] = -kBox; A.y[3] = kBox;  A.lab[3] = -1;
    // scan 1: the kNear nearest charges by float32 distance; clipping with them
    // nearest first cuts the square down to (nearly) the cell in a few steps,
    // so the polygon stays small (a far-first order can grow it by one vertex
    // per clip)
    float kd[kNear];
    int kj[kNear];
    int kn = 0;
    float thr = 3.0e38f;
    for (int64_t t0 = 0; t0 < n; t0 += kOrdThreads) {
        const int64_t js = t0 + tid;
        tile[tid] = js < n ? posf[js] : make_float2(3.0e18f, 3.0e18f);
        __syncthreads();
        if (act) {
            const int cnt = (int)min((int64_t)kOrdThreads, n - t0);
            for (int jj = 0; jj < cnt; ++jj) {
                const float2 q = tile[jj];
                const float ex = q.x - rf.x, ey = q.y - rf.y;
                const float d2 = fmaf(ex, ex, ey * ey);
                const int64_t j = t0 + jj;
                if (d2 >= thr || j == i) continue;
                int p = kn < kNear ? kn++ : kNear - 1;
                while (p > 0 && kd[p - 1] > d2) { kd[p] = kd[p - 1]; kj[p] = kj[p - 1]; --p; }
                kd[p] = d2;
                kj[p] = (int)j;
                if (kn == kNear) thr = kd[kNear - 1];
            }
        }
        __syncthreads();
    }
    if (act) {
        for (int w = 0; w < kn; ++w) {
            const double2 q = pos[kj[w]];
            if (q.x == r.x && q.y == r.y) { coincident = true; continue; }
            if (clip(*cur, *nxt, r, q, kj[w], &overflow)) { Poly* t = cur; cur = nxt; nxt = t; }
        }
    }
    // scan 2: every charge that can still cut the cell
    float lim = reject_limit(far2(*cur, r));
    for (int64_t t0 = 0; t0 < n; t0 += kOrdThreads) {
        const int64_t js = t0 + tid;
        tile[tid] = js < n ? posf[js] : make_float2(3.0e18f, 3.0e18f);
        __syncthreads();
        if (act) {
            const int cnt = (int)min((int64_t)kOrdThreads, n - t0);
            for (int jj = 0; jj < cnt; ++jj) {
                const float2 q = tile[jj];
                const float ex = q.x - rf.x, ey = q.y - rf.y;
                if (fmaf(ex, ex, ey * ey) >= lim) continue;
                const int64_t j = t0 + jj;
                if (j == i) continue;
                const double2 qd = pos[j];
                if (qd.x == r.x && qd.y == r.y) { coincident = true; continue; }
                if (clip(*cur, *nxt, r, qd, (int)j, &overflow)) {
                    Poly* t = cur; cur = nxt; nxt = t;
                    lim = reject_limit(far2(*cur, r));
                }
            }
        }
        __syncthreads();
    }
    if (!act) return;
    if (overflow) set_status(st, ST_INVALID);
    if (coincident) set_status(st, ST_NONFINITE);
    // neighbours: the distinct labels on the cell's edges, ascending
    int nb[kMaxPoly];
    int cnt = 0;
    for (int k = 0; k < cur->nv; ++k) {
        const int l = cur->lab[k];
        if (l < 0) continue;
        bool dup = false;
        for (int q = 0; q < cnt; ++q) dup |= nb[q] == l;
        if (dup) continue;
        int p = cnt++;
        while (p > 0 && nb[p - 1] > l) { nb[p] = nb[p - 1]; --p; }
        nb[p] = l;
    }
    z[i] = cnt;
    // psi6: mean of the sixth power of the unit bond vectors, as complex numbers
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < cnt; ++q) {
        const double2 p = pos[nb[q]];
        const double dx = p.x - r.x, dy = p.y - r.y;
        const double a2 = dx * dx - dy * dy, b2 = 2.0 * dx * dy;   // (dx + i dy)^2
        const double a3 = a2 * dx - b2 * dy, b3 = a2 * dy + b2 * dx; // ^3
        const double a6 = a3 * a3 - b3 * b3, b6 = 2.0 * a3 * b3;    // ^6
        const double d2 = dx * dx + dy * dy, d6 = d2 * d2 * d2;
        sr += a6 / d6;
        si += b6 / d6;
    }
    psi[i] = cnt > 0 ? make_double2(sr / cnt, si / cnt) : make_double2(0.0, 0.0);
    if (nbr) {
        if (cnt > max_nbr) set_status(st, ST_INVALID);
        for (int q = 0; q < max_nbr; ++q) nbr[i * max_nbr + q] = q < cnt ? nb[q] : -1;
    }
}

// <|psi6|>, |<psi6>| and P(z): one CTA, counts by shared atomics (order-free),
// sums in double-double in a fixed tree order.
__global__ void __launch_bounds__(1024) k_order_summary(const int32_t* __restrict__ z, const double2* __restrict__ psi,
                                                        int64_t n, double* __restrict__ out)
{
    __shared__ unsigned long long hist[kZBins];
    __shared__ double sh[1024];
    const int tid = threadIdx.x;
    if (tid < kZBins) hist[tid] = 0ull;
    __syncthreads();
    double ah = 0.0, al = 0.0, rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
    for (int64_t i = tid; i < n; i += 1024) {
        const double2 p = psi[i];
        dd_add(ah, al, sqrt(p.x * p.x + p.y * p.y));
        dd_add(rh, rl, p.x);
        dd_add(ih, il, p.y);
        atomicAdd(&hist[min(z[i], kZBins - 1)], 1ull);
    }
    double v[3] = {ah + al, rh + rl, ih + il};
    for (int k = 0; k < 3; ++k) v[k] = block_sum<1024>(v[k], sh);
    __syncthreads();
    if (tid == 0) {
        const double inv = n > 0 ? 1.0 / (double)n : 0.0;
        out[0] = v[0] * inv;
        out[1] = sqrt(v[1] * v[1] + v[2] * v[2]) * inv;
        for (int k = 0; k < kZBins; ++k) out[2 + k] = (double)hist[k] * inv;
    }
}

}  // namespace

}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_voronoi_order(const double* pos, int64_t n, int32_t* z, double* psi6, int32_t* nbr, int32_t max_nbr,
                           double* summary, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_voronoi_order");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0 || n > INT32_MAX || (n > 0 && (!pos || !z || !psi6)) || (nbr && max_nbr < 1) ||
        (reinterpret_cast<uintptr_t>(pos) & 15) || (reinterpret_cast<uintptr_t>(psi6) & 15) ||
        (reinterpret_cast<uintptr_t>(summary) & 7))
        return TC_ERR_INVALID_ARG;
    tc_status err = TC_OK;
    int* st = device_status(&err);
    if (!st) return err;
    if (n == 0) {
        if (summary) return cuda_status(cudaMemsetAsync(summary, 0, sizeof(double) * (2 + kZBins), s));
        return TC_OK;
    }
    Carver c;
    c.take<float2>(n);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    float2* posf = c.take<float2>(n);
    const double2* p2 = reinterpret_cast<const double2*>(pos);
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8L * sm_count()));
    k_to_float2<<<nb, 256, 0, s>>>(p2, n, posf);
    k_voronoi<<<(unsigned)((n + kOrdThreads - 1) / kOrdThreads), kOrdThreads, 0, s>>>(
        p2, posf, n, z, reinterpret_cast<double2*>(psi6), nbr, max_nbr, st);
    if (summary) k_order_summary<<<1, 1024, 0, s>>>(z, reinterpret_cast<const double2*>(psi6), n, summary);
    return cuda_status(cudaGetLastError(), "structure analysis launch");
}

}  // extern "C"
