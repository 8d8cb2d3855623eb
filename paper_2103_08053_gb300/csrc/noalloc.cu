// noalloc.cu -- tc_count_dag_noalloc: counting an oriented graph without
// allocating any device memory.
//
// Some callers cannot call cudaMalloc: their device memory is entirely held
// by another allocator (a framework's caching pool that reserves the GPU up
// front), or they run a latency-critical loop where an allocation -- which may
// synchronise the whole device -- is not acceptable. For them this entry point
// runs the same binning and counting kernels as tc_count_dag, with the kernels'
// scratch (queue counters, the warp-worker list and its descriptors, the
// thread-block work items) in the file-scope array g_noalloc_scratch below.
// The array is part of the library image: every GPU that loads the library
// holds its kScratchBytes (about 5.8 MB) until the process exits.
#include <mutex>

#include "api_internal.h"

namespace {

using tcg::CountCfg;
using tcg::DevCounters;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int64_t kMaxN = TC_NOALLOC_MAX_N;
constexpr int64_t kMaxM = TC_NOALLOC_MAX_M;
// This entry point always runs with the default parameters, so binning makes
// at most item_capacity(n, m, default item_neighbors) thread-block work items
// (one per large vertex plus one per item_neighbors of its out-edges).
constexpr int64_t kItemCap = tcg::item_capacity(kMaxN, kMaxM, tcg::DEFAULT_ITEM_NEIGHBORS);

// scratch layout: counters | warp-worker list | its descriptors | block items
constexpr size_t kOffCtr = 0;
constexpr size_t kOffList = align256(sizeof(DevCounters));
constexpr size_t kOffDesc = kOffList + align256((size_t)(kMaxN + 1) * sizeof(int32_t));
constexpr size_t kOffItems = kOffDesc + align256((size_t)(kMaxN + 1) * sizeof(int2));
constexpr size_t kScratchBytes = kOffItems + align256((size_t)kItemCap * sizeof(int2));

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device set-up, done once by the first call on each device (with that
// device current): the device address of the scratch array and the launch
// configuration for the default parameters.
struct DeviceSetup {
    bool done = false;
    unsigned char* scratch = nullptr;
    int num_sms = 0;
    CountCfg cfg{};
};
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

tc_status setup_device(int dev, DeviceSetup** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tcg::cuda_status(nullptr, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return tcg::cuda_status(nullptr, e, "cudaDeviceGetAttribute");
        tc_params prm;
        CountCfg cfg;
        tc_status st = tcg::resolve_params(nullptr, nullptr, &prm, &cfg);
        if (st) return st;
        e = tcg::count_kernel_setup(cfg, sms);
        if (e != cudaSuccess) return tcg::cuda_status(nullptr, e, "count kernel setup");
        s.scratch = static_cast<unsigned char*>(p);
        s.num_sms = sms;
        s.cfg = cfg;
        s.done = true;
    }
    *out = &s;
    return TC_OK;
}

}  // namespace

size_t tcg::noalloc_scratch_bytes() { return kScratchBytes; }

extern "C" tc_status tc_count_dag_noalloc(const tc_dag* dag, uint64_t* count_device, int32_t* error_device,
                                          void* stream) {
    if (!dag || !count_device) return tcg::ctx_fail(nullptr, TC_ERR_INVALID_ARG, "dag and count_device are required");
    if (dag->n < 0 || dag->m < 0 || (dag->n > 0 && !dag->dag_ptr) || (dag->m > 0 && !dag->dag_col))
        return tcg::ctx_fail(nullptr, TC_ERR_INVALID_ARG, "bad tc_dag");
    if (dag->n > kMaxN || dag->m > kMaxM)
        return tcg::ctx_fail(nullptr, TC_ERR_UNSUPPORTED,
                             "tc_count_dag_noalloc: graph exceeds the static scratch (n %lld > %lld or m %lld > %lld)",
                             (long long)dag->n, (long long)kMaxN, (long long)dag->m, (long long)kMaxM);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tcg::cuda_status(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return tcg::ctx_fail(nullptr, TC_ERR_UNSUPPORTED, "device index too large");
    DeviceSetup* s = nullptr;
    tc_status st = setup_device(dev, &s);
    if (st) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevCounters* ctr = reinterpret_cast<DevCounters*>(s->scratch + kOffCtr);
    int32_t* list = reinterpret_cast<int32_t*>(s->scratch + kOffList);
    int2* desc = reinterpret_cast<int2*>(s->scratch + kOffDesc);
    int2* items = reinterpret_cast<int2*>(s->scratch + kOffItems);
    long long launches = 0;
    // the counters (queue cursors, list sizes, total, error bits) must start at zero
    e = cudaMemsetAsync(ctr, 0, sizeof(DevCounters), cs);
    if (e == cudaSuccess && dag->n > 0) {
        e = tcg::launch_bin(dag->dag_ptr, dag->n, s->cfg, list, desc, items, kItemCap, ctr, s->num_sms, cs,
                            &launches);
        if (e == cudaSuccess)
            e = tcg::launch_count(dag->dag_ptr, dag->dag_col, dag->n, list, desc, items, nullptr, s->cfg, ctr, cs,
                                  &launches);
    }
    if (e == cudaSuccess)
        e = tcg::launch_finish(ctr, reinterpret_cast<unsigned long long*>(count_device), error_device, cs, &launches);
    return tcg::cuda_status(nullptr, e, "tc_count_dag_noalloc kernels");
}
