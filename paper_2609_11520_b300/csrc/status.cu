// Status and error-message plumbing of the C ABI.
#include <cstring>

#include "common.cuh"

namespace fio {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fio_status fail(fio_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

fio_status cuda_status(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA;
}

struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_pool;
static size_t g_pool_used = 0;

static cudaEvent_t pool_event() {
    if (g_pool_used == g_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_pool.push_back(e);
    }
    return g_pool[g_pool_used++];
}

bool profiling_enabled() { return g_prof_on; }

void prof_begin(const char* name, cudaStream_t st) {
    ProfRec r{name, pool_event(), pool_event()};
    cudaEventRecord(r.a, st);
    g_prof.push_back(r);
}

void prof_end(cudaStream_t st) {
    if (!g_prof.empty()) cudaEventRecord(g_prof.back().b, st);
}

}  // namespace fio

extern "C" const char* fio_last_error(void) { return fio::g_last_error.c_str(); }

extern "C" fio_status fio_profile_enable(int on) {
    fio::g_prof_on = on != 0;
    return FIO_OK;
}

extern "C" fio_status fio_profile_report(char* buf, int64_t len) {
    using namespace fio;
    if (!buf || len <= 0) return fail(FIO_EINVAL, "fio_profile_report: no buffer");
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<long> cnt;
    for (auto& r : g_prof) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_status(e, "fio_profile_report");
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        size_t i = 0;
        while (i < names.size() && names[i] != r.name) ++i;
        if (i == names.size()) {
            names.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[i] += t;
        cnt[i] += 1;
    }
    std::string out;
    for (size_t i = 0; i < names.size(); ++i)
        out += names[i] + " " + std::to_string(cnt[i]) + " " + std::to_string(ms[i]) + "\n";
    g_prof.clear();
    g_pool_used = 0;
    if (int64_t(out.size()) + 1 > len) return fail(FIO_EINVAL, "fio_profile_report: buffer too small");
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return FIO_OK;
}
