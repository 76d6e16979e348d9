// Kernel tracing and launch counting.
//
// When tracing is on, every kernel launch of the library is bracketed by two
// CUDA events recorded on the stream it is launched on, and each public
// operation by another pair; fides_trace_read() synchronises those events and
// reports launches and total device time per name.  The launch counter counts
// every kernel the library launches, traced or not.
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "fides_internal.cuh"

namespace {

struct Rec {
    const char *name;
    int e0, e1;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_events;
size_t g_next = 0;
std::vector<Rec> g_recs;
unsigned long long g_launches = 0;

int take_event()
{
    if (g_next == g_events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        g_events.push_back(e);
    }
    return (int)g_next++;
}

}  // namespace

int fides_trace_begin(const char *name, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    int e0 = take_event(), e1 = take_event();
    if (e0 < 0 || e1 < 0) return -1;
    cudaEventRecord(g_events[e0], st);
    g_recs.push_back(Rec{name, e0, e1});
    return (int)g_recs.size() - 1;
}

void fides_trace_end(int id, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (id < 0 || (size_t)id >= g_recs.size()) return;
    cudaEventRecord(g_events[g_recs[id].e1], st);
}

void fides_count_launch()
{
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launches;
}

extern "C" int fides_trace_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return FIDES_OK;
}

extern "C" void fides_trace_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.clear();
    g_next = 0;
}

extern "C" uint64_t fides_kernel_launches(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_launches;
}

extern "C" int fides_trace_read(fides_trace_stat *out, int max, int *n_out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!n_out || (max > 0 && !out)) return fides_set_error(FIDES_ERR_ARG, "fides_trace_read: bad arguments");
    std::vector<std::string> order;
    std::unordered_map<std::string, fides_trace_stat> agg;
    for (const Rec &r : g_recs) {
        cudaError_t e = cudaEventSynchronize(g_events[r.e1]);
        if (e != cudaSuccess) return fides_check_cuda(e, "fides_trace_read");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, g_events[r.e0], g_events[r.e1]);
        if (e != cudaSuccess) return fides_check_cuda(e, "fides_trace_read");
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            it = agg.emplace(r.name, fides_trace_stat{r.name, 0, 0.0}).first;
        }
        it->second.launches += 1;
        it->second.total_ms += ms;
    }
    int n = 0;
    for (const std::string &k : order) {
        if (n < max) out[n] = agg[k];
        ++n;
    }
    *n_out = n;
    return FIDES_OK;
}

// Sets the tracing state and returns the previous one (used to keep event
// records out of captured graphs).
int fides_trace_set(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const int was = g_on ? 1 : 0;
    g_on = on != 0;
    return was;
}
