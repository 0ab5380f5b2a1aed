// tc_api.cu -- status codes, per-device status word, per-stream workspace.
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "tc_plan.cuh"

namespace tc {

int g_mixed_config = 0;


namespace {

struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
};

std::mutex g_mu;
std::map<std::tuple<int, cudaStream_t, int>, Block> g_ws;
std::map<int, int*> g_status;
std::map<int, cudaStream_t> g_cap;

thread_local std::string g_last_error;

constexpr size_t kExecCacheMax = 8;  // executable graphs kept per device

// An executable graph and the signature of the graph it was made from: per
// node its type and, for a kernel node, the kernel, grid and block.  Only an
// executable graph with the same signature is updated in place, so an update
// changes kernel arguments and nothing else.
struct CachedExec {
    cudaGraphExec_t exec;
    std::vector<uintptr_t> sig;
};
std::mutex g_exec_mu;
std::map<int, std::vector<CachedExec>> g_exec;  // most recently returned last
thread_local std::vector<uintptr_t> g_taken_sig;  // signature of the graph last handed out on this thread

bool graph_signature(cudaGraph_t g, std::vector<uintptr_t>& sig)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return false;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return false;
    sig.clear();
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(node, &t) != cudaSuccess) return false;
        sig.push_back((uintptr_t)t);
        if (t == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess) return false;
            sig.push_back((uintptr_t)kp.func);
            sig.push_back(((uintptr_t)kp.gridDim.x << 32) | ((uintptr_t)kp.gridDim.y << 16) | kp.gridDim.z);
            sig.push_back(((uintptr_t)kp.blockDim.x << 32) | ((uintptr_t)kp.blockDim.y << 16) | kp.blockDim.z);
        }
    }
    return true;
}

}  // namespace

cudaGraphExec_t take_graph_exec(cudaGraph_t graph, cudaError_t* e)
{
    int dev = 0;
    if ((*e = cudaGetDevice(&dev)) != cudaSuccess) return nullptr;
    g_taken_sig.clear();
    if (graph_signature(graph, g_taken_sig)) {
        std::lock_guard<std::mutex> lk(g_exec_mu);
        auto& v = g_exec[dev];
        for (size_t i = v.size(); i-- > 0;) {
            if (v[i].sig != g_taken_sig) continue;
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(v[i].exec, graph, &info) == cudaSuccess) {
                cudaGraphExec_t x = v[i].exec;
                v.erase(v.begin() + (std::ptrdiff_t)i);
                return x;
            }
            cudaGetLastError();  // refused: instantiate below
        }
    } else {
        cudaGetLastError();
        g_taken_sig.clear();
    }
    cudaGraphExec_t x = nullptr;
    *e = cudaGraphInstantiate(&x, graph, 0);
    return *e == cudaSuccess ? x : nullptr;
}

void give_graph_exec(cudaGraphExec_t exec)
{
    if (!exec) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || g_taken_sig.empty()) {
        cudaGraphExecDestroy(exec);
        return;
    }
    std::lock_guard<std::mutex> lk(g_exec_mu);
    auto& v = g_exec[dev];
    v.push_back(CachedExec{exec, g_taken_sig});
    if (v.size() > kExecCacheMax) {
        cudaGraphExecDestroy(v.front().exec);
        v.erase(v.begin());
    }
}

void release_graph_execs()
{
    std::lock_guard<std::mutex> lk(g_exec_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : g_exec) {
        cudaSetDevice(kv.first);
        for (const CachedExec& x : kv.second) cudaGraphExecDestroy(x.exec);
    }
    g_exec.clear();
    cudaSetDevice(cur);
}

tc_status cuda_fail(cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return TC_OK;
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    g_last_error = buf;
    return TC_ERR_CUDA;
}

void set_last_error(const char* msg)
{
    g_last_error = msg;
}

void* workspace(cudaStream_t s, size_t bytes, tc_status* err, int slot)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *err = TC_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    Block& b = g_ws[{dev, s, slot}];
    if (b.bytes >= bytes && b.ptr) return b.ptr;
    size_t want = align_up(bytes + bytes / 4, size_t(2) << 20);
    if (b.ptr) {
        // no kernel of this stream may still use the old block
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaFree(b.ptr) != cudaSuccess) {
            *err = TC_ERR_CUDA;
            return nullptr;
        }
        b.ptr = nullptr;
        b.bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        *err = TC_ERR_NO_MEMORY;
        return nullptr;
    }
    // counters used by the last-block reductions must start at zero
    if (cudaMemsetAsync(p, 0, want, s) != cudaSuccess) {
        cudaFree(p);
        *err = TC_ERR_CUDA;
        return nullptr;
    }
    b.ptr = p;
    b.bytes = want;
    return p;
}

int* device_status(tc_status* err)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *err = TC_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_status.find(dev);
    if (it != g_status.end()) return it->second;
    int* p = nullptr;
    if (cudaMalloc(&p, 256) != cudaSuccess || cudaMemset(p, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        *err = TC_ERR_NO_MEMORY;
        return nullptr;
    }
    g_status[dev] = p;
    return p;
}

cudaStream_t capture_stream(tc_status* err)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *err = TC_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cap.find(dev);
    if (it != g_cap.end()) return it->second;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        *err = TC_ERR_CUDA;
        return nullptr;
    }
    g_cap[dev] = cs;
    return cs;
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace tc

extern "C" {

const char* tc_status_string(tc_status s)
{
    switch (s) {
        case TC_OK: return "ok";
        case TC_ERR_INVALID_ARG: return "invalid argument";
        case TC_ERR_CUDA: return "CUDA runtime error";
        case TC_ERR_NONFINITE: return "non-finite result (coincident charges or NaN)";
        case TC_ERR_OUTSIDE_DISK: return "charge outside the disk";
        case TC_ERR_TIMEOUT: return "bounded device wait expired";
        case TC_ERR_NOT_CONVERGED: return "not converged";
        case TC_ERR_NO_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

int32_t tc_pass_config_count(tc_precision prec)
{
    return prec == TC_MIXED ? tc::kMixedConfigs : ((prec == TC_FP64 || prec == TC_F64X) ? 1 : 0);
}

tc_status tc_set_pass_config(tc_precision prec, int32_t config)
{
    if (prec == TC_MIXED && config >= 0 && config < tc::kMixedConfigs) {
        tc::g_mixed_config = config;
        return TC_OK;
    }
    if ((prec == TC_FP64 || prec == TC_F64X) && config == 0) return TC_OK;
    return TC_ERR_INVALID_ARG;
}

int32_t tc_get_pass_config(tc_precision prec)
{
    return prec == TC_MIXED ? tc::g_mixed_config : 0;
}

const char* tc_last_error(void)
{
    return tc::g_last_error.c_str();
}

tc_status tc_sync_status(tc_stream stream)
{
    tc_status err = TC_OK;
    int* st = tc::device_status(&err);
    if (!st) return err;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaError_t e_ = cudaStreamSynchronize(s); e_ != cudaSuccess) return tc::cuda_fail(e_, "cudaStreamSynchronize");
    int h = 0;
    if (cudaError_t e_ = cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost); e_ != cudaSuccess) return tc::cuda_fail(e_, "cudaMemcpy");
    if (h != 0 && cudaMemset(st, 0, sizeof(int)) != cudaSuccess) return TC_ERR_CUDA;
    return static_cast<tc_status>(h);
}

void tc_shutdown(void)
{
    std::lock_guard<std::mutex> lk(tc::g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : tc::g_ws) {
        cudaSetDevice(std::get<0>(kv.first));
        cudaStreamSynchronize(std::get<1>(kv.first));
        cudaFree(kv.second.ptr);
    }
    tc::g_ws.clear();
    for (auto& kv : tc::g_status) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second);
    }
    tc::g_status.clear();
    for (auto& kv : tc::g_cap) {
        cudaSetDevice(kv.first);
        cudaStreamDestroy(kv.second);
    }
    tc::g_cap.clear();
    cudaSetDevice(cur);
    tc::release_graph_execs();
}

}  // extern "C"
