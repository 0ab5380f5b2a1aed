// tc_cycle.cu -- the adaptive optimisation cycle of Sec. II C on the GPU.
//
// Step 2 (local-energy statistics and the defect list) runs in one CTA; step 3
// (the centre) and the zone of step 4 (the m charges nearest to the centre)
// run one CTA per subdomain: an exact radix select of the m-th smallest
// (d^2, index) key over all n charges, then an ordered compaction that lists
// the zone in ascending index.  The cycle driver strings these together with
// the all-pairs local energies (step 1) and the batched relaxation with its
// sequential float64 accept (step 4).
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_plan.cuh"

static_assert(sizeof(tc_zone_params) == 48, "tc_zone_params layout");
static_assert(sizeof(tc_cycle_params) == 184, "tc_cycle_params layout");

namespace tc {

namespace {

constexpr int kStatThreads = 1024;
constexpr int kSelThreads = 512;
constexpr double kPi = 3.14159265358979323846;

struct ZoneArgs {
    double p_defect;
    double radius;
    int64_t m_min, m_max, period, phase;
};

// Zone size at schedule position q: a triangle wave between m_min (q = 0 mod
// period) and m_max (q = period/2 mod period), capped at n.  Integer
// arithmetic only, so host and device agree exactly.
__host__ __device__ __forceinline__ int64_t zone_size(int64_t q, int64_t m_min, int64_t m_max, int64_t period,
                                                      int64_t n)
{
    const int64_t qq = q % period;
    const int64_t tri = qq < period - qq ? qq : period - qq;
    const int64_t m = m_min + (2 * (m_max - m_min) * tri) / period;
    return m < n ? m : n;
}

// Squared distance rounded as written (two products, one sum, no fused
// multiply-add); a non-negative double orders like its bit pattern.
__device__ __forceinline__ unsigned long long dist_key(double2 p, double2 c)
{
    const double dx = __dsub_rn(p.x, c.x), dy = __dsub_rn(p.y, c.y);
    return (unsigned long long)__double_as_longlong(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// Exclusive prefix count of `flag` over the CTA in thread order; *total gets
// the CTA's count.  Every thread of the CTA must call it.
template <int THREADS> __device__ __forceinline__ int block_excl_count(int flag, int* warp_tot, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_tot[w] = __popc(b);
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < THREADS / 32; ++k) {
        const int c = warp_tot[k];
        before += k < w ? c : 0;
        tot += c;
    }
    *total = tot;
    __syncthreads();
    return before + __popc(b & ((1u << lane) - 1u));
}

// Double-double CTA sum of per-thread (hi, lo) partials, combined in a fixed
// tree order (deterministic).
template <int THREADS> __device__ double block_dd_sum(double hi, double lo, double* sh_hi, double* sh_lo)
{
    sh_hi[threadIdx.x] = hi;
    sh_lo[threadIdx.x] = lo;
    __syncthreads();
#pragma unroll
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double h = sh_hi[threadIdx.x], l = sh_lo[threadIdx.x];
            dd_add(h, l, sh_hi[threadIdx.x + w]);
            sh_hi[threadIdx.x] = h;
            sh_lo[threadIdx.x] = l + sh_lo[threadIdx.x + w];
        }
        __syncthreads();
    }
    const double r = sh_hi[0] + sh_lo[0];
    __syncthreads();
    return r;
}

// Step 2: mu, sigma_e (population) of e over all n, and the defect list
// D = { i : e_i > mu + kappa sigma_e, |r_i|^2 < rin2, not pinned } in ascending i.
// stats = (mu, sigma_e, |D|).  One CTA.
__global__ void __launch_bounds__(kStatThreads) k_zone_stats(const double2* __restrict__ pos,
                                                             const double* __restrict__ e,
                                                             const uint8_t* __restrict__ flags, int64_t n,
                                                             double kappa, double rin2, int32_t* __restrict__ D,
                                                             double* __restrict__ stats)
{
    __shared__ double sh_hi[kStatThreads], sh_lo[kStatThreads];
    __shared__ int warp_tot[32];
    const int tid = threadIdx.x;
    double hi = 0.0, lo = 0.0;
    for (int64_t i = tid; i < n; i += kStatThreads) dd_add(hi, lo, e[i]);
    const double mu = block_dd_sum<kStatThreads>(hi, lo, sh_hi, sh_lo) / (double)n;
    hi = lo = 0.0;
    for (int64_t i = tid; i < n; i += kStatThreads) {
        const double d = __dsub_rn(e[i], mu);
        dd_add(hi, lo, __dmul_rn(d, d));
    }
    const double sigma = sqrt(block_dd_sum<kStatThreads>(hi, lo, sh_hi, sh_lo) / (double)n);
    const double thr = __dadd_rn(mu, __dmul_rn(kappa, sigma));
    int64_t base = 0;
    for (int64_t c0 = 0; c0 < n; c0 += kStatThreads) {
        const int64_t i = c0 + tid;
        int flag = 0;
        if (i < n) {
            const double2 p = pos[i];
            const double r2 = __dadd_rn(__dmul_rn(p.x, p.x), __dmul_rn(p.y, p.y));
            flag = (e[i] > thr) && (r2 < rin2) && !(flags && flags[i]);
        }
        int tot = 0;
        const int r = block_excl_count<kStatThreads>(flag, warp_tot, &tot);
        if (flag) D[base + r] = (int32_t)i;
        base += tot;
    }
    if (tid == 0) {
        stats[0] = mu;
        stats[1] = sigma;
        stats[2] = (double)base;
    }
}

// Step 3 and the zone of step 4 for subdomain s = blockIdx.x (fixed, nullable,
// replaces the drawn centres).
__global__ void __launch_bounds__(kSelThreads) k_zone_select(const double2* __restrict__ pos, int64_t n,
                                                             const int32_t* __restrict__ D,
                                                             const double* __restrict__ stats,
                                                             const double* __restrict__ uni,
                                                             const double2* __restrict__ fixed, ZoneArgs z,
                                                             int32_t* __restrict__ idx, int64_t* __restrict__ offsets,
                                                             double2* __restrict__ centres)
{
    __shared__ unsigned hist[256];
    __shared__ int warp_tot[32];
    __shared__ int64_t red[kSelThreads / 32];
    __shared__ double2 s_c;
    __shared__ unsigned s_bin;
    __shared__ int64_t s_k;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t m = zone_size(z.phase + s, z.m_min, z.m_max, z.period, n);

    // offset of this zone: the sizes of the zones before it
    int64_t part = 0;
    for (int64_t t = tid; t < s; t += kSelThreads) part += zone_size(z.phase + t, z.m_min, z.m_max, z.period, n);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_down_sync(0xffffffffu, part, d);
    if (lane == 0) red[w] = part;
    if (tid == 0) {
        double2 c;
        if (fixed) {
            c = fixed[s];
        } else if (uni[3 * s] < z.p_defect && (int64_t)stats[2] > 0) {
            const double u1 = uni[3 * s + 1];
            const int64_t nd = (int64_t)stats[2];
            int64_t k = (int64_t)__dmul_rn(u1, (double)nd);
            k = k > nd - 1 ? nd - 1 : (k < 0 ? 0 : k);
            c = pos[D[k]];
        } else {
            const double u1 = uni[3 * s + 1], u2 = uni[3 * s + 2];
            const double r = __dmul_rn(sqrt(u1), z.radius), t = __dmul_rn(2.0 * kPi, u2);
            double sn, cs;
            sincos(t, &sn, &cs);
            c = make_double2(__dmul_rn(r, cs), __dmul_rn(r, sn));
        }
        s_c = c;
        if (centres) centres[s] = c;
    }
    __syncthreads();
    int64_t off = 0;
#pragma unroll
    for (int k = 0; k < kSelThreads / 32; ++k) off += red[k];
    if (tid == 0) {
        offsets[s + 1] = off + m;
        if (s == 0) offsets[0] = 0;
    }
    if (m <= 0) return;
    const double2 c = s_c;
    int32_t* out = idx + off;
    if (m >= n) {
        for (int64_t i = tid; i < n; i += kSelThreads) out[i] = (int32_t)i;
        return;
    }

    // radix select, 8 bits per pass from the top: after the passes `prefix`
    // is the m-th smallest key and k the number of keys equal to it that the
    // zone takes (the smallest indices among them)
    unsigned long long prefix = 0ull, mask = 0ull;
    int64_t k = m;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += kSelThreads) hist[b] = 0u;
        __syncthreads();
        for (int64_t c0 = 0; c0 < n; c0 += kSelThreads) {
            const int64_t i = c0 + tid;
            bool in = false;
            unsigned bin = 256u + (unsigned)lane;  // distinct per lane: never matches a real bin
            if (i < n) {
                const unsigned long long key = dist_key(pos[i], c);
                in = (key & mask) == prefix;
                if (in) bin = (unsigned)(key >> shift) & 255u;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (w == 0) {
            unsigned cnt[8], sum = 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                cnt[j] = hist[8 * lane + j];
                sum += cnt[j];
            }
            unsigned incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            const int64_t excl = (int64_t)(incl - sum);
            if (excl < k && k <= (int64_t)incl) {
                int64_t kk = k - excl;
                int j = 0;
                while (j < 7 && kk > (int64_t)cnt[j]) {
                    kk -= cnt[j];
                    ++j;
                }
                s_bin = 8u * (unsigned)lane + (unsigned)j;
                s_k = kk;
            }
        }
        __syncthreads();
        prefix |= (unsigned long long)s_bin << shift;
        mask |= 255ull << shift;
        k = s_k;
        __syncthreads();
    }

    // ordered compaction: keys below the m-th, then the first k equal to it
    const unsigned long long kstar = prefix;
    const int64_t need_eq = k;
    int64_t less_base = 0, eq_base = 0;
    for (int64_t c0 = 0; c0 < n; c0 += kSelThreads) {
        const int64_t i = c0 + tid;
        int fl = 0, fe = 0;
        if (i < n) {
            const unsigned long long key = dist_key(pos[i], c);
            fl = key < kstar;
            fe = key == kstar;
        }
        int tl = 0, te = 0;
        const int rl = block_excl_count<kSelThreads>(fl, warp_tot, &tl);
        const int re = block_excl_count<kSelThreads>(fe, warp_tot, &te);
        const int64_t eq_rank = eq_base + re;
        if (fl || (fe && eq_rank < need_eq))
            out[less_base + rl + (eq_rank < need_eq ? eq_rank : need_eq)] = (int32_t)i;
        less_base += tl;
        eq_base += te;
    }
}

// Border-interior split: every charge is a boundary charge except the listed
// interior ones; then the projection (pinned to the unit circle, the others
// confined to sigma).
__global__ void k_border_flags(const int32_t* __restrict__ interior, int64_t m, uint8_t* __restrict__ flags)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        flags[interior[k]] = 0;
}

__global__ void k_border_project(double2* __restrict__ pos, int64_t n, double sigma, const uint8_t* __restrict__ flags)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pos[i] = project1(pos[i], sigma, flags[i] != 0);
}

tc_status check_zone(const tc_zone_params* z)
{
    if (!z || z->m_min < 0 || z->m_max < z->m_min || z->period < 1 || z->phase < 0 || !(z->radius > 0.0) ||
        !std::isfinite(z->radius) || !(z->wall_tol >= 0.0) || !(z->wall_tol < z->radius) ||
        !std::isfinite(z->kappa) || !(z->p_defect >= 0.0 && z->p_defect <= 1.0)) {
        set_last_error("zone parameters: need 0 <= m_min <= m_max, period >= 1, phase >= 0, radius > 0, "
                       "0 <= wall_tol < radius, finite kappa, 0 <= p_defect <= 1");
        return TC_ERR_INVALID_ARG;
    }
    return TC_OK;
}

ZoneArgs zone_args(const tc_zone_params* z, int64_t phase)
{
    ZoneArgs a;
    a.p_defect = z->p_defect;
    a.radius = z->radius;
    a.m_min = z->m_min;
    a.m_max = z->m_max;
    a.period = z->period;
    a.phase = phase;
    return a;
}

// Host-side offsets of n_sub zones starting at schedule position phase.
void zone_offsets(const tc_zone_params* z, int64_t phase, int64_t n, int32_t n_sub, int64_t* offsets)
{
    offsets[0] = 0;
    for (int32_t s = 0; s < n_sub; ++s)
        offsets[s + 1] = offsets[s] + zone_size(phase + s, z->m_min, z->m_max, z->period, n);
}

// Steps 2-3 and the zones; the defect list lives in the slot-0 workspace.
tc_status select_zones(const double* pos, int64_t n, const double* local_e, const uint8_t* flags,
                       const tc_zone_params* z, double radius, int64_t phase, int32_t n_sub, const double* uniforms,
                       int32_t* idx, int64_t* offsets, double* centres, double* stats, cudaStream_t s)
{
    tc_status err = TC_OK;
    Carver c;
    c.take<int32_t>(n);
    c.take<double>(4);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    int32_t* D = c.take<int32_t>(n);
    double* st = c.take<double>(4);
    if (!stats) stats = st;
    const double rin = radius - z->wall_tol;
    const double2* p2 = reinterpret_cast<const double2*>(pos);
    ZoneArgs za = zone_args(z, phase);
    za.radius = radius;
    k_zone_stats<<<1, kStatThreads, 0, s>>>(p2, local_e, flags, n, z->kappa, rin * rin, D, stats);
    k_zone_select<<<(unsigned)n_sub, kSelThreads, 0, s>>>(p2, n, D, stats, uniforms, nullptr, za, idx, offsets,
                                                         reinterpret_cast<double2*>(centres));
    return cuda_status(cudaGetLastError(), "zone selection launch");
}

bool misaligned(const void* p, uintptr_t a)
{
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0;
}

// Length of the longest prefix of pairwise disjoint zones among zones 0 .. k-1
// (at least 1) into *out.  One CTA walks the zones in order, testing a zone's
// charges against a bit map of the charges taken so far and adding them when
// none is; `taken` (n bits) must be zero on entry.
constexpr int kPrefixThreads = 1024;

__global__ void __launch_bounds__(kPrefixThreads) k_disjoint_prefix(const int32_t* __restrict__ idx,
                                                                     const int64_t* __restrict__ offs, int32_t k,
                                                                     uint32_t* __restrict__ taken, int32_t* out)
{
    __shared__ int clash;
    int32_t s = 0;
    for (; s < k; ++s) {
        if (threadIdx.x == 0) clash = 0;
        __syncthreads();
        const int64_t a = offs[s], b = offs[s + 1];
        for (int64_t i = a + threadIdx.x; i < b; i += kPrefixThreads) {
            const int32_t j = idx[i];
            if ((taken[j >> 5] >> (j & 31)) & 1u) clash = 1;
        }
        __syncthreads();
        if (clash) break;
        for (int64_t i = a + threadIdx.x; i < b; i += kPrefixThreads) {
            const int32_t j = idx[i];
            atomicOr(&taken[j >> 5], 1u << (j & 31));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s > 0 ? s : 1;
}

}  // namespace

// Eq. sigma (Sec. II B): the initial radius of the interior charges, 1 - 1/(2 sqrt(N)).
inline double eq_sigma(int64_t n) { return 1.0 - 0.5 / std::sqrt((double)n); }

}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_zone_offsets(const tc_zone_params* prm, int64_t n, int32_t n_sub, int64_t* offsets)
{
    tc_status err = check_zone(prm);
    if (err != TC_OK) return err;
    if (n < 0 || n_sub < 0 || !offsets) return TC_ERR_INVALID_ARG;
    zone_offsets(prm, prm->phase, n, n_sub, offsets);
    return TC_OK;
}

tc_status tc_select_subdomains(const double* pos, int64_t n, const double* local_e, const uint8_t* flags,
                               const tc_zone_params* prm, int32_t n_sub, const double* uniforms, int32_t* idx,
                               int64_t* offsets, double* centres, double* stats, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_select_subdomains");
    tc_status err = check_zone(prm);
    if (err != TC_OK) return err;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0 || n_sub < 0 || !offsets || misaligned(offsets, 8)) return TC_ERR_INVALID_ARG;
    if (n_sub == 0) return cuda_status(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s), "cudaMemsetAsync");
    if (n < 1 || n > INT32_MAX || !pos || !local_e || !uniforms || misaligned(pos, 16) || misaligned(local_e, 8) ||
        misaligned(uniforms, 8) || misaligned(idx, 4) || misaligned(centres, 16) || misaligned(stats, 8))
        return TC_ERR_INVALID_ARG;
    if (!idx) {
        // idx may be null only when every zone is empty
        std::vector<int64_t> off(n_sub + 1);
        zone_offsets(prm, prm->phase, n, n_sub, off.data());
        if (off[n_sub] > 0) return TC_ERR_INVALID_ARG;
    }
    return select_zones(pos, n, local_e, flags, prm, prm->radius, prm->phase, n_sub, uniforms, idx, offsets, centres,
                        stats, s);
}

tc_status tc_cycle(double* pos, int64_t n, const uint8_t* flags, const tc_cycle_params* prm, int32_t n_sub,
                   const double* uniforms, tc_subdomain_result* out, double* energy, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_cycle");
    if (!prm) return TC_ERR_INVALID_ARG;
    tc_status err = check_zone(&prm->zone);
    if (err != TC_OK) return err;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const tc_precision lp = static_cast<tc_precision>(prm->local_precision);
    // sigma0 <= 0 asks for the initial interior radius of Eq. sigma
    const double sigma0 = prm->sigma0 <= 0.0 && n >= 1 ? eq_sigma(n) : prm->sigma0;
    if (n_sub < 0 || prm->batch < 1 || (lp != TC_FP64 && lp != TC_MIXED) || misaligned(energy, 8) ||
        !(sigma0 > prm->zone.wall_tol) || !(sigma0 <= prm->sigma1) || !(prm->sigma1 <= 1.0)) {
        set_last_error("tc_cycle: need n_sub >= 0, batch >= 1, a valid local_precision and "
                       "wall_tol < sigma0 <= sigma1 <= 1");
        return TC_ERR_INVALID_ARG;
    }
    if (n_sub == 0) return TC_OK;
    if (n < 1 || n > INT32_MAX || !pos || !uniforms || !out || misaligned(pos, 16) || misaligned(uniforms, 8) ||
        misaligned(out, 8))
        return TC_ERR_INVALID_ARG;
    const int32_t B = std::min(prm->batch, n_sub);
    // the sigma ramp runs over the whole cycle: subdomains ramp_first .. of ramp_total
    const int64_t total = prm->ramp_total > 0 ? prm->ramp_total : n_sub;
    const int64_t first = prm->ramp_total > 0 ? prm->ramp_first : 0;
    if (first < 0 || first + n_sub > total || (prm->disjoint == 0 && first % prm->batch != 0)) {
        set_last_error("tc_cycle: need 0 <= ramp_first, ramp_first + n_sub <= ramp_total, and (fixed batches) "
                       "ramp_first a multiple of batch");
        return TC_ERR_INVALID_ARG;
    }
    const int32_t Bt = std::min<int64_t>(prm->batch, total);
    const int64_t n_batches = (total + Bt - 1) / Bt;  // of the whole cycle (fixed batches)
    const int64_t b_first = first / Bt;
    if (prm->disjoint != 0 && prm->disjoint != 1) {
        set_last_error("tc_cycle: disjoint must be 0 or 1");
        return TC_ERR_INVALID_ARG;
    }
    const bool disjoint = prm->disjoint == 1;
    // the largest batch's zones fix the buffer sizes (disjoint batches may start at any subdomain)
    int64_t cap = 0;
    std::vector<int64_t> off(B + 1);
    for (int64_t b0 = 0; b0 < n_sub; b0 += disjoint ? 1 : B) {
        const int32_t k = (int32_t)std::min<int64_t>(B, n_sub - b0);
        zone_offsets(&prm->zone, prm->zone.phase + b0, n, k, off.data());
        cap = std::max(cap, off[k]);
    }
    const int64_t taken_words = disjoint ? (n + 31) / 32 : 0;
    Carver c;
    c.take<double>(n);
    c.take<int32_t>(std::max<int64_t>(cap, 1));
    c.take<int64_t>(B + 1);
    c.take<double>(1);
    c.take<uint32_t>(taken_words);
    c.take<int32_t>(1);
    void* ws = workspace(s, c.off, &err, 1);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    double* e_loc = c.take<double>(n);
    int32_t* idx = c.take<int32_t>(std::max<int64_t>(cap, 1));
    int64_t* offs = c.take<int64_t>(B + 1);
    double* e_tot = c.take<double>(1);
    uint32_t* taken = c.take<uint32_t>(taken_words);
    int32_t* prefix = c.take<int32_t>(1);

    tc_relax_params rp = prm->relax;
    rp.accept = 1;
    int64_t b = 0;
    for (int64_t b0 = 0, k = 0; b0 < n_sub; b0 += k, ++b) {
        k = std::min<int64_t>(B, n_sub - b0);
        // interior radius of this batch: linear ramp sigma0 -> sigma1 over the batches (fixed
        // batches) or over the subdomain index of the batch's first zone (disjoint batches)
        double sigma;
        if (!disjoint)
            sigma = n_batches <= 1 ? prm->sigma1
                                   : sigma0 + (prm->sigma1 - sigma0) * (double)(b_first + b) / (double)(n_batches - 1);
        else
            sigma = total <= 1 ? prm->sigma1
                               : sigma0 + (prm->sigma1 - sigma0) * (double)(first + b0) / (double)(total - 1);
        rp.radius = sigma;
        err = allpairs(pos, n, lp, nullptr, energy ? energy + b : e_tot, e_loc, s);
        if (err != TC_OK) return err;
        err = select_zones(pos, n, e_loc, flags, &prm->zone, sigma, prm->zone.phase + b0, (int32_t)k,
                           uniforms + 3 * b0, idx, offs, nullptr, nullptr, s);
        if (err != TC_OK) return err;
        if (disjoint && k > 1) {
            int32_t kk = 1;
            cudaError_t e = cudaMemsetAsync(taken, 0, 4 * (size_t)taken_words, s);
            if (e == cudaSuccess) {
                k_disjoint_prefix<<<1, kPrefixThreads, 0, s>>>(idx, offs, (int32_t)k, taken, prefix);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&kk, prefix, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "disjoint prefix");
            if (kk < 1 || kk > k) return TC_ERR_CUDA;
            k = kk;
        }
        err = relax(pos, n, idx, offs, (int32_t)k, nullptr, flags, &rp, out + b0, s);
        if (err != TC_OK) return err;
    }
    if (energy) return allpairs(pos, n, lp, nullptr, energy + b, nullptr, s);
    return TC_OK;
}

int64_t tc_boundary_count(int64_t n)
{
    if (n <= 0) return 0;
    const double c = std::cbrt((double)n);
    const double nb = 2.84328 * c * c - 0.530196 * c - 2.32866;
    const int64_t k = (int64_t)std::floor(nb + 0.5);
    return k < 0 ? 0 : (k > n ? n : k);
}

tc_status tc_border_split(double* pos, int64_t n, int64_t n_b, double sigma, uint8_t* flags, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_border_split");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (sigma <= 0.0 && n >= 1) sigma = eq_sigma(n);  // Eq. sigma
    if (n < 0 || n > INT32_MAX || n_b < 0 || n_b > n || !(sigma > 0.0) || !(sigma <= 1.0) ||
        (n > 0 && (!pos || !flags)) || misaligned(pos, 16))
        return TC_ERR_INVALID_ARG;
    if (n == 0) return TC_OK;
    tc_status err = TC_OK;
    const int64_t m = n - n_b;  // interior charges: the m nearest to the centre
    Carver c;
    c.take<int32_t>(std::max<int64_t>(m, 1));
    c.take<int64_t>(2);
    c.take<double2>(1);
    c.take<double>(4);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    int32_t* interior = c.take<int32_t>(std::max<int64_t>(m, 1));
    int64_t* offs = c.take<int64_t>(2);
    double2* origin = c.take<double2>(1);
    double* stats = c.take<double>(4);
    ZoneArgs za{};
    za.p_defect = 0.0;
    za.radius = 1.0;
    za.m_min = za.m_max = m;
    za.period = 1;
    za.phase = 0;
    cudaError_t e = cudaMemsetAsync(origin, 0, sizeof(double2), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, 4 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 1, (size_t)n, s);
    if (e != cudaSuccess) return cuda_fail(e, "border split set-up");
    double2* p2 = reinterpret_cast<double2*>(pos);
    k_zone_select<<<1, kSelThreads, 0, s>>>(p2, n, nullptr, stats, nullptr, origin, za, interior, offs, nullptr);
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8L * sm_count()));
    if (m > 0) k_border_flags<<<nb, 256, 0, s>>>(interior, m, flags);
    k_border_project<<<nb, 256, 0, s>>>(p2, n, sigma, flags);
    return cuda_status(cudaGetLastError(), "border split launch");
}

}  // extern "C"
