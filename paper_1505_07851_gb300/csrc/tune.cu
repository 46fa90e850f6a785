// Autotuner cache (see tune.h).
#include <map>
#include <mutex>
#include <tuple>

#include "context.h"
#include "tune.h"

namespace pcm {

namespace {
struct Entry {
    int choice;
    float ms[3];
};
std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, Entry> g_table;
}  // namespace

int tune_bucket(long long n)
{
    int b = 0;
    while (n > 1) {
        n >>= 1;
        ++b;
    }
    return b;
}

int tune_get(int device, int kind, int L, int bucket)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(std::make_tuple(device, kind, L, bucket));
    return it == g_table.end() ? -1 : it->second.choice;
}

void tune_set(int device, int kind, int L, int bucket, int choice, float ms0, float ms1, float ms2)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[std::make_tuple(device, kind, L, bucket)] = Entry{choice, {ms0, ms1, ms2}};
}

int tune_table(int *out, int max)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int n = 0;
    for (const auto &kv : g_table) {
        if (n < max && out) {
            int *o = out + 8 * n;
            o[0] = std::get<0>(kv.first);
            o[1] = std::get<1>(kv.first);
            o[2] = std::get<2>(kv.first);
            o[3] = std::get<3>(kv.first);
            o[4] = kv.second.choice;
            for (int v = 0; v < 3; ++v) o[5 + v] = (int)(1000.f * kv.second.ms[v] + 0.5f);
        }
        ++n;
    }
    return n;
}

}  // namespace pcm

extern "C" int pcm_autotune_table(int *entries, int max_entries)
{
    return pcm::tune_table(entries, max_entries);
}
