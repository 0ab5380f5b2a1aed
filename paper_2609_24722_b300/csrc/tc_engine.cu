// tc_engine.cu -- libtc entry points: energy, gradient, projection, pairwise
// energy change and the batched subdomain / instance relaxation.
//
// Every entry point funnels into the generic pair pass (tc_pass.cuh): a
// "problem" is a set of moving rows plus a source list (a snapshot range of
// the configuration with the problem's own charges masked out, followed by
// the problem's own rows).  The all-pairs energy of Eq. (hamiltonian) is one
// problem whose rows are all N charges; an independent instance is one
// problem per configuration; a subdomain of Sec. II D is one problem whose
// rows are its active set A and whose snapshot is the fixed set F.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc_plan.cuh"

namespace tc {

__global__ void k_split(const double2* __restrict__ pos, int64_t n, float4* __restrict__ out, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y))
            set_status(st, ST_NONFINITE);
        else if (!inside(p.x, p.y))
            set_status(st, ST_OUTSIDE);
        out[i] = split4(p.x, p.y);
    }
}

__global__ void k_split3(const double2* __restrict__ pos, int64_t n, fx3* __restrict__ out, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y))
            set_status(st, ST_NONFINITE);
        else if (!inside(p.x, p.y))
            set_status(st, ST_OUTSIDE);
        out[i] = split3(p.x, p.y);
    }
}

__global__ void k_check(const double2* __restrict__ pos, int64_t n, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y))
            set_status(st, ST_NONFINITE);
        else if (!inside(p.x, p.y))
            set_status(st, ST_OUTSIDE);
    }
}

// Finish of the all-pairs pass: per row, add the slots in order, then (after a
// symmetric float64 pass, col_e non-null) the source sums that row blocks
// rb < t / 2 left for the row's tile t, in order of rb; write grad and local
// energies; the last block adds the block energies in order.
template <bool WANT_G>
__global__ void k_finish_allpairs(Prob p, int64_t W, int64_t G, const double* __restrict__ part_e,
                                  const double2* __restrict__ part_g, const double* __restrict__ col_e,
                                  const double2* __restrict__ col_g, double2* __restrict__ grad,
                                  double* __restrict__ local_e, double* __restrict__ block_e,
                                  unsigned* __restrict__ counter, double* __restrict__ energy, int* st)
{
    __shared__ double sh[256];
    __shared__ bool last;
    const int64_t n = p.m;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        int rb = (int)(i / kRB);
        int64_t c = slot_count(p, rb, 0, W, G);
        double eh = 0.0, el = 0.0;
        double gx = 0.0, gy = 0.0;
        for (int64_t s = 0; s < c; ++s) {
            dd_add(eh, el, part_e[s * n + i]);
            if (WANT_G) {
                double2 q = part_g[s * n + i];
                gx += q.x;
                gy += q.y;
            }
        }
        if (col_e) {
            const int64_t nb = i / kT / 2;
            for (int64_t b = 0; b < nb; ++b) {
                dd_add(eh, el, col_e[b * n + i]);
                if (WANT_G) {
                    const double2 q = col_g[b * n + i];
                    gx += q.x;
                    gy += q.y;
                }
            }
        }
        e = eh + el;
        if (!isfinite(e) || !isfinite(gx) || !isfinite(gy)) set_status(st, ST_NONFINITE);
        if (local_e) local_e[i] = e;
        if (WANT_G) grad[i] = make_double2(gx, gy);
    }
    double b = block_sum<256>(e, sh);
    if (threadIdx.x == 0) {
        block_e[blockIdx.x] = b;
        __threadfence();
        unsigned done = atomicAdd(counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double hi = 0.0, lo = 0.0;
        if (threadIdx.x == 0) {
            for (unsigned k = 0; k < gridDim.x; ++k) dd_add(hi, lo, ((volatile double*)block_e)[k]);
            if (energy) *energy = hi + lo;
            if (!isfinite(hi + lo)) set_status(st, ST_NONFINITE);
            *counter = 0u;
        }
    }
}

__global__ void k_project(double2* __restrict__ pos, int64_t n, double radius, const uint8_t* __restrict__ flags)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = pos[i];
        double r = sqrt(__dadd_rn(__dmul_rn(p.x, p.x), __dmul_rn(p.y, p.y)));
        if (flags && flags[i]) {
            if (r > 0.0) pos[i] = make_double2(p.x / r, p.y / r);
        } else if (r > radius) {
            double s = radius / r;
            pos[i] = make_double2(__dmul_rn(p.x, s), __dmul_rn(p.y, s));
        }
    }
}

// ------------------------------------------------------------ all pairs ---

tc_status allpairs(const double* pos, int64_t n, tc_precision prec, double* grad, double* energy,
                          double* local_e, cudaStream_t s)
{
    if (n < 0 || (n > 0 && !pos) || (prec != TC_FP64 && prec != TC_MIXED && prec != TC_F64X)) return TC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos) & 15) || (grad && (reinterpret_cast<uintptr_t>(grad) & 15)) ||
        (energy && (reinterpret_cast<uintptr_t>(energy) & 7)) || (local_e && (reinterpret_cast<uintptr_t>(local_e) & 7)))
        return TC_ERR_INVALID_ARG;
    tc_status err = TC_OK;
    int* st = device_status(&err);
    if (!st) return err;
    if (n <= 1) {
        cudaError_t e = cudaSuccess;
        if (energy) e = cudaMemsetAsync(energy, 0, sizeof(double), s);
        if (e == cudaSuccess && grad && n > 0) e = cudaMemsetAsync(grad, 0, 16 * n, s);
        if (e == cudaSuccess && local_e && n > 0) e = cudaMemsetAsync(local_e, 0, 8 * n, s);
        if (e == cudaSuccess && n == 1) {
            k_check<<<1, 32, 0, s>>>(reinterpret_cast<const double2*>(pos), n, st);
            e = cudaGetLastError();
        }
        return cuda_status(e);
    }
    Plan P;
    Prob p{};
    p.row_base = 0;
    p.snap_b = p.snap_e = 0;
    p.mask_off = -1;
    p.m = (int32_t)n;
    P.prob.push_back(p);
    plan_units(P);
    const bool want_g = grad != nullptr;
    int64_t G;
    if (prec == TC_MIXED)
        G = want_g ? pass_grid<PASS_MIXED, true, true>(P.W) : pass_grid<PASS_MIXED, true, false>(P.W);
    else if (prec == TC_F64X)
        G = want_g ? pass_grid<PASS_F64X, true, true>(P.W) : pass_grid<PASS_F64X, true, false>(P.W);
    else
        G = want_g ? pass_grid<PASS_F64, true, true>(P.W) : pass_grid<PASS_F64, true, false>(P.W);
    // the mixed and float64 passes: ranges from a queue (mixed_ranges), the same for every launch
    // shape; the float64 pass takes each unordered pair once when its source sums (24 bytes per
    // charge and row block) fit 2 GiB
    const int64_t ctas = G;
    const bool sym = prec == TC_FP64 && (int64_t)P.prob[0].n_rb * n * 24 <= (int64_t(2) << 30);
    if (prec == TC_MIXED) G = mixed_ranges(P.W);
    if (sym) G = sym_ranges(P.W);
    P.G = G;
    P.slots = plan_slots(P.prob, 0, 1, 0, P.W, G);
    const int64_t nb = (n + 255) / 256;
    const int64_t ncol = sym ? (int64_t)P.prob[0].n_rb * n : 0;

    Carver c;
    c.take<float4>(prec == TC_MIXED ? n : 0);
    c.take<fx3>(prec == TC_F64X ? n : 0);
    c.take<double>(P.slots * n);
    c.take<double2>(want_g ? P.slots * n : 0);
    c.take<double>(nb);
    c.take<double>(ncol);
    c.take<double2>(want_g ? ncol : 0);
    void* ws = workspace(s, c.off, &err);
    if (!ws) return err;
    c.base = static_cast<char*>(ws);
    c.off = kCounterBytes;
    float4* split = c.take<float4>(prec == TC_MIXED ? n : 0);
    fx3* split3v = c.take<fx3>(prec == TC_F64X ? n : 0);
    double* part_e = c.take<double>(P.slots * n);
    double2* part_g = c.take<double2>(want_g ? P.slots * n : 0);
    double* block_e = c.take<double>(nb);
    double* col_e = sym ? c.take<double>(ncol) : nullptr;
    double2* col_g = sym && want_g ? c.take<double2>(ncol) : nullptr;
    unsigned* counter = reinterpret_cast<unsigned*>(ws);

    PassArgs a{};
    a.prob = nullptr;
    a.single = P.prob[0];
    a.S = 1;
    a.W = P.W;
    a.M = n;
    a.mask = nullptr;
    a.active = nullptr;
    a.part_e = part_e;
    a.part_g = part_g;
    const double2* pos2 = reinterpret_cast<const double2*>(pos);
    cudaError_t e;
    int cb = (int)std::min<int64_t>(nb, 4L * sm_count());
    if (prec == TC_MIXED) {
        k_split<<<cb, 256, 0, s>>>(pos2, n, split, st);
        a.rows = split;
        a.snap = split;
        a.ticket = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kPassCtrOff);
        a.ctas = mixed_ctas(G, ctas);
        if ((e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s)) != cudaSuccess) return cuda_fail(e, "set-up");
        e = want_g ? launch_pass<PASS_MIXED, true, true>(a, G, 0, 0, s)
                   : launch_pass<PASS_MIXED, true, false>(a, G, 0, 0, s);
    } else if (prec == TC_F64X) {
        k_split3<<<cb, 256, 0, s>>>(pos2, n, split3v, st);
        a.rows = split3v;
        a.snap = split3v;
        e = want_g ? launch_pass<PASS_F64X, true, true>(a, G, 0, 0, s)
                   : launch_pass<PASS_F64X, true, false>(a, G, 0, 0, s);
    } else {
        k_check<<<cb, 256, 0, s>>>(pos2, n, st);
        a.rows = pos2;
        a.snap = pos2;
        if (sym) {
            a.sym = 1;
            a.col_e = col_e;
            a.col_g = col_g;
            a.col_stride = n;
            a.ticket = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kPassCtrOff);
            a.ctas = mixed_ctas(G, want_g ? pass_grid<PASS_F64, true, true, true>(P.W)
                                          : pass_grid<PASS_F64, true, false, true>(P.W));
            if ((e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s)) != cudaSuccess) return cuda_fail(e, "set-up");
        }
        e = want_g ? launch_pass<PASS_F64, true, true>(a, G, 0, 0, s)
                   : launch_pass<PASS_F64, true, false>(a, G, 0, 0, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "set-up");
    if (want_g)
        k_finish_allpairs<true><<<(unsigned)nb, 256, 0, s>>>(P.prob[0], P.W, G, part_e, part_g, col_e, col_g,
                                                             reinterpret_cast<double2*>(grad), local_e, block_e,
                                                             counter, energy, st);
    else
        k_finish_allpairs<false><<<(unsigned)nb, 256, 0, s>>>(P.prob[0], P.W, G, part_e, nullptr, col_e, nullptr,
                                                              nullptr, local_e, block_e, counter, energy, st);
    return cuda_status(cudaGetLastError());
}

}  // namespace tc

extern "C" {

tc_status tc_energy(const double* pos, int64_t n, tc_precision prec, double* energy, double* local_e,
                    tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_energy");
    if (!energy) return TC_ERR_INVALID_ARG;
    return tc::allpairs(pos, n, prec, nullptr, energy, local_e, reinterpret_cast<cudaStream_t>(stream));
}

tc_status tc_grad(const double* pos, int64_t n, tc_precision prec, double* grad, double* energy, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_grad");
    if (!grad) return TC_ERR_INVALID_ARG;
    return tc::allpairs(pos, n, prec, grad, energy, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

tc_status tc_project_disk(double* pos, int64_t n, double radius, const uint8_t* flags, tc_stream stream)
{
    tc::NvtxRange nvtx_range("tc_project_disk");
    if (n < 0 || (n > 0 && !pos) || !(radius > 0.0) || (reinterpret_cast<uintptr_t>(pos) & 15))
        return TC_ERR_INVALID_ARG;
    if (n == 0) return TC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int nb = (int)std::min<int64_t>((n + 255) / 256, 8L * tc::sm_count());
    tc::k_project<<<nb, 256, 0, s>>>(reinterpret_cast<double2*>(pos), n, radius, flags);
    return tc::cuda_status(cudaGetLastError());
}

}  // extern "C"
