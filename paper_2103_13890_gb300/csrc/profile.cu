// Optional per-kernel-class timing with CUDA events recorded on the launching
// stream around each stencil launch (off by default; jfnk_profile_enable).
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace jfnk {

namespace {
struct Rec {
    int cls;
    cudaEvent_t a, b;
};
struct ClassInfo {
    std::string name;
    double work;  // elements processed per launch
};
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_pool_next = 0;
std::vector<ClassInfo> g_classes;
std::map<std::string, int> g_index;
int g_open = -1;

cudaEvent_t take_event() {
    if (g_pool_next == g_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_pool.push_back(e);
    }
    return g_pool[g_pool_next++];
}
}  // namespace

bool prof_on() { return g_on; }

void prof_begin(const char* name, double work, cudaStream_t st) {
    if (!g_on) return;
    auto it = g_index.find(name);
    int cls;
    if (it == g_index.end()) {
        cls = (int)g_classes.size();
        g_classes.push_back({name, work});
        g_index[name] = cls;
    } else {
        cls = it->second;
    }
    Rec r{cls, take_event(), take_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    g_open = (int)g_recs.size() - 1;
}

void prof_end(cudaStream_t st) {
    if (!g_on || g_open < 0) return;
    cudaEventRecord(g_recs[g_open].b, st);
    g_open = -1;
}

}  // namespace jfnk

using namespace jfnk;

void jfnk_profile_enable(int on) {
    g_on = on != 0;
    g_recs.clear();
    g_classes.clear();
    g_index.clear();
    g_pool_next = 0;
    g_open = -1;
}

int jfnk_profile_read(int max_classes, char* names, int name_len, long long* launches, double* total_ms,
                      double* work_per_launch) {
    cudaDeviceSynchronize();
    const int nc = (int)g_classes.size();
    std::vector<long long> cnt(nc, 0);
    std::vector<double> ms(nc, 0.0);
    for (const Rec& r : g_recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            cnt[r.cls]++;
            ms[r.cls] += t;
        }
    }
    const int n = nc < max_classes ? nc : max_classes;
    for (int i = 0; i < n; ++i) {
        if (names) {
            strncpy(names + (size_t)i * name_len, g_classes[i].name.c_str(), name_len - 1);
            names[(size_t)i * name_len + name_len - 1] = 0;
        }
        if (launches) launches[i] = cnt[i];
        if (total_ms) total_ms[i] = ms[i];
        if (work_per_launch) work_per_launch[i] = g_classes[i].work;
    }
    return nc;
}
