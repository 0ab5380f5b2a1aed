// tc_noalloc.cu -- total energy without any device allocation.
//
// tc_energy keeps its scratch (hi/lo split of the positions, per-row partial
// sums, per-block sums, a counter) in a workspace it grows with cudaMalloc.
// tc_energy_noalloc computes the same energy with the same pair kernels, but
// its scratch is one fixed array in the library's device image, so the call
// never allocates.  That array exists on every GPU that loads libtc and stays
// there until the process exits.
#include <mutex>

#include "tc_plan.cuh"

namespace tc {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB on every device that loads libtc
constexpr int64_t kStaticMaxN = 200000;                   // largest n accepted (fits the array)

// The scratch itself.  Bytes [0, 256) hold the last-block counter and a
// status word; the split positions, row partials and block sums follow.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device.  In host code
// the name g_static_scratch is only a host-side stand-in for the symbol, not
// a device address, so it is never passed to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_base[kMaxDevices] = {};

tc_status scratch_base(void** out)
{
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        if (cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch); e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return TC_OK;
}

// Checks every charge (finite, inside the disk) and writes the hi/lo split
// when `split` is not null.
__global__ void k_noalloc_prep(const double2* __restrict__ pos, int64_t n, float4* __restrict__ split, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = pos[i];
        if (!isfinite(p.x) || !isfinite(p.y))
            set_status(st, ST_NONFINITE);
        else if (!inside(p.x, p.y))
            set_status(st, ST_OUTSIDE);
        if (split) split[i] = split4(p.x, p.y);
    }
}

// Adds each row's slots in order (local energies), then the block sums in
// order in the last block.  Any device-side error makes the energy NaN.
__global__ void k_noalloc_finish(Prob p, int64_t W, int64_t G, const double* __restrict__ part_e,
                                 double* __restrict__ local_e, double* __restrict__ block_e,
                                 unsigned* __restrict__ counter, int* st, double* __restrict__ energy)
{
    __shared__ double sh[256];
    __shared__ bool last;
    const int64_t n = p.m;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        const int64_t c = slot_count(p, (int)(i / kRB), 0, W, G);
        double hi = 0.0, lo = 0.0;
        for (int64_t k = 0; k < c; ++k) dd_add(hi, lo, part_e[k * n + i]);
        e = hi + lo;
        if (!isfinite(e)) set_status(st, ST_NONFINITE);
        if (local_e) local_e[i] = e;
    }
    const double b = block_sum<256>(e, sh);
    if (threadIdx.x == 0) {
        block_e[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double hi = 0.0, lo = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) dd_add(hi, lo, ((volatile double*)block_e)[k]);
        *energy = (*((volatile int*)st) != 0) ? __longlong_as_double(0x7ff8000000000000LL) : hi + lo;
        *counter = 0u;
    }
}

// n = 1: no pairs, so E = 0 and e_0 = 0, unless the one charge is invalid (NaN energy).
__global__ void k_noalloc_one(const int* st, double* __restrict__ energy, double* __restrict__ local_e)
{
    *energy = (*((volatile const int*)st) != 0) ? __longlong_as_double(0x7ff8000000000000LL) : 0.0;
    if (local_e) *local_e = 0.0;
}

}  // namespace

static tc_status energy_noalloc(const double* pos, int64_t n, tc_precision prec, double* energy, double* local_e,
                                cudaStream_t s)
{
    tc::NvtxRange nvtx_range("tc_energy_noalloc");
    if (n < 0 || (n > 0 && !pos) || !energy || (prec != TC_FP64 && prec != TC_MIXED)) return TC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos) & 15) || (reinterpret_cast<uintptr_t>(energy) & 7) ||
        (reinterpret_cast<uintptr_t>(local_e) & 7))
        return TC_ERR_INVALID_ARG;
    if (n > kStaticMaxN) {
        set_last_error("tc_energy_noalloc: n exceeds the static scratch limit of 200000 charges");
        return TC_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    if (tc_status st0 = scratch_base(&base); st0 != TC_OK) return st0;
    unsigned* counter = static_cast<unsigned*>(base);
    int* st = reinterpret_cast<int*>(static_cast<char*>(base) + 4);
    // counter and status word start at zero on every call
    if (cudaError_t e = cudaMemsetAsync(base, 0, kCounterBytes, s); e != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync (static scratch)");
    const double2* pos2 = reinterpret_cast<const double2*>(pos);
    if (n == 0) {
        if (cudaError_t e = cudaMemsetAsync(energy, 0, sizeof(double), s); e != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync");
        return TC_OK;
    }
    if (n == 1) {
        // the one charge is still checked, as tc_energy checks it
        k_noalloc_prep<<<1, 32, 0, s>>>(pos2, 1, nullptr, st);
        k_noalloc_one<<<1, 1, 0, s>>>(st, energy, local_e);
        return cuda_status(cudaGetLastError(), "tc_energy_noalloc launch");
    }
    Plan P;
    Prob p{};
    p.snap_b = p.snap_e = 0;
    p.mask_off = -1;
    p.m = (int32_t)n;
    P.prob.push_back(p);
    plan_units(P);
    const int64_t G = prec == TC_MIXED ? pass_grid<PASS_MIXED, true, false>(P.W) : pass_grid<PASS_F64, true, false>(P.W);
    const int64_t slots = plan_slots(P.prob, 0, 1, 0, P.W, G);
    const int64_t nb = (n + 255) / 256;
    Carver c;
    c.base = static_cast<char*>(base);
    float4* split = c.take<float4>(prec == TC_MIXED ? n : 0);
    double* part_e = c.take<double>(slots * n);
    double* block_e = c.take<double>(nb);
    if (c.off > kStaticScratchBytes) {
        set_last_error("tc_energy_noalloc: this n needs more than the 16 MiB static scratch");
        return TC_ERR_INVALID_ARG;
    }
    const int cb = (int)std::min<int64_t>(nb, 4L * sm_count());
    k_noalloc_prep<<<cb, 256, 0, s>>>(pos2, n, prec == TC_MIXED ? split : nullptr, st);
    PassArgs a{};
    a.prob = nullptr;
    a.single = P.prob[0];
    a.S = 1;
    a.W = P.W;
    a.M = n;
    a.rows = prec == TC_MIXED ? static_cast<const void*>(split) : static_cast<const void*>(pos2);
    a.snap = a.rows;
    a.part_e = part_e;
    cudaError_t e = prec == TC_MIXED ? launch_pass<PASS_MIXED, true, false>(a, G, 0, 0, s)
                                     : launch_pass<PASS_F64, true, false>(a, G, 0, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "tc_energy_noalloc pass launch");
    k_noalloc_finish<<<(unsigned)nb, 256, 0, s>>>(P.prob[0], P.W, G, part_e, local_e, block_e, counter, st, energy);
    return cuda_status(cudaGetLastError(), "tc_energy_noalloc launch");
}

}  // namespace tc

extern "C" tc_status tc_energy_noalloc(const double* pos, int64_t n, tc_precision prec, double* energy,
                                       double* local_e, tc_stream stream)
{
    return tc::energy_noalloc(pos, n, prec, energy, local_e, reinterpret_cast<cudaStream_t>(stream));
}
