// Per-kernel CUDA-event timing and launch counting behind tmd_profile_*.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tmd_internal.cuh"

namespace tmd {

namespace {

struct Pending {
    int kernel;
    cudaEvent_t start, stop;
};

struct Registry {
    std::mutex mu;
    bool on = false;
    std::vector<std::string> names;
    std::vector<int64_t> launches;
    std::vector<double> ms;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int64_t total_launches = 0;

    int id(const char *name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.emplace_back(name);
        launches.push_back(0);
        ms.push_back(0.0);
        return (int)names.size() - 1;
    }
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

Registry &reg() {
    static Registry r;
    return r;
}

}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s) : stream_(s), kernel_(-1), start_(nullptr) {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.total_launches++;
    if (!r.on) return;
    kernel_ = r.id(name);
    start_ = r.take();
    cudaEventRecord(start_, s);
}

ProfScope::~ProfScope() {
    if (kernel_ < 0) return;
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    cudaEvent_t stop = r.take();
    cudaEventRecord(stop, stream_);
    r.pending.push_back({kernel_, start_, stop});
}

bool profiling_on() {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    return r.on;
}

void add_launches(int64_t k) {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.total_launches += k;
}

}  // namespace tmd

using namespace tmd;

extern "C" {

tmd_status tmd_profile_enable(int32_t on) {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.on = on != 0;
    return TMD_OK;
}

tmd_status tmd_profile_read(tmd_kernel_stat *out, int32_t cap, int32_t *count, int32_t reset) {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    for (Pending &p : r.pending) {
        cudaError_t e = cudaEventSynchronize(p.stop);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        cudaEventElapsedTime(&t, p.start, p.stop);
        r.launches[p.kernel]++;
        r.ms[p.kernel] += t;
        r.pool.push_back(p.start);
        r.pool.push_back(p.stop);
    }
    r.pending.clear();
    int32_t n = 0;
    for (size_t i = 0; i < r.names.size(); ++i) {
        if (r.launches[i] == 0) continue;
        if (out && n < cap) {
            std::memset(out[n].name, 0, sizeof(out[n].name));
            std::strncpy(out[n].name, r.names[i].c_str(), sizeof(out[n].name) - 1);
            out[n].launches = r.launches[i];
            out[n].total_ms = r.ms[i];
        }
        ++n;
    }
    if (count) *count = n;
    if (reset)
        for (size_t i = 0; i < r.names.size(); ++i) {
            r.launches[i] = 0;
            r.ms[i] = 0.0;
        }
    return TMD_OK;
}

int64_t tmd_launch_count(void) {
    Registry &r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    return r.total_launches;
}

}  // extern "C"
