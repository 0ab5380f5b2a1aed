// tc_internal.h -- host-side helpers shared by the libtc translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/tc.h"

namespace tc {

// Per-(device, stream, slot) scratch workspace.  Grows with cudaMalloc (after
// a stream synchronisation, so no in-flight kernel uses the old block) and is
// freed by tc_shutdown().  Slot 0 is the per-call scratch of every entry
// point; slot 1 holds buffers that must outlive the calls a driver makes in
// sequence (the cycle's zones).  Returns nullptr and sets *err on failure.
void* workspace(cudaStream_t s, size_t bytes, tc_status* err, int slot = 0);

// Per-device status word (device int), allocated on first use.
int* device_status(tc_status* err);

// Per-device private non-blocking stream used only to capture CUDA graphs
// (the legacy default stream cannot be captured).
cudaStream_t capture_stream(tc_status* err);

// Executable step-loop graphs kept across calls, per device.  take_graph_exec
// returns an executable graph for `graph`: a cached one updated in place with
// cudaGraphExecUpdate when one has the same shape (only kernel arguments
// differ), else a new instantiation (nullptr and *e set on failure).  The
// caller owns it until give_graph_exec returns it to the cache (the cache
// keeps a few per device and destroys the rest).  release_graph_execs
// destroys every cached one (tc_shutdown).
cudaGraphExec_t take_graph_exec(cudaGraph_t graph, cudaError_t* e);
void give_graph_exec(cudaGraphExec_t exec);
void release_graph_execs();

// SM count and current device.
int sm_count();

// Record a failed CUDA runtime call (name and error text, per host thread)
// for tc_last_error() and return TC_ERR_CUDA; TC_OK for cudaSuccess.
tc_status cuda_fail(cudaError_t e, const char* where);

inline tc_status cuda_status(cudaError_t e, const char* where = "CUDA call") { return cuda_fail(e, where); }

// Set the text tc_last_error() returns for this host thread.
void set_last_error(const char* msg);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NVTX range around one public call (visible to ncu --nvtx and other
// profilers; costs nothing when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// The first kCounterBytes of every workspace hold zero-initialised counters
// for last-block reductions (each user resets its counter to zero); the rest
// is carved per call.
constexpr size_t kCounterBytes = 256;

// Bump allocator over a workspace block: take<T>(n) returns the next 256-byte
// aligned region of n elements, after the counter area.
struct Carver {
    char* base = nullptr;
    size_t off = kCounterBytes;
    template <class T> T* take(size_t count)
    {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Entry points reused by the cycle driver (same contracts as tc_energy /
// tc_grad and tc_relax_subdomains).
tc_status allpairs(const double* pos, int64_t n, tc_precision prec, double* grad, double* energy,
                   double* local_e, cudaStream_t s);
tc_status relax(double* pos, int64_t n, const int32_t* idx, const int64_t* offsets, int32_t n_sub,
                const int64_t* world, const uint8_t* flags, const tc_relax_params* prm,
                tc_subdomain_result* out, cudaStream_t s);

}  // namespace tc
