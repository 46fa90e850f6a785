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
    float ms0, ms1;
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

void tune_set(int device, int kind, int L, int bucket, int choice, float ms0, float ms1)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[std::make_tuple(device, kind, L, bucket)] = Entry{choice, ms0, ms1};
}

int tune_table(int *out, int max)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int n = 0;
    for (const auto &kv : g_table) {
        if (n < max && out) {
            out[5 * n + 0] = std::get<0>(kv.first);
            out[5 * n + 1] = std::get<1>(kv.first);
            out[5 * n + 2] = std::get<2>(kv.first);
            out[5 * n + 3] = std::get<3>(kv.first);
            out[5 * n + 4] = kv.second.choice;
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
