// Online tuning: the learned-cost-model search of Section IV-B spread over
// the library's own calls instead of run up front.
//
// With online tuning on, a call that passes no plan and finds no tuned plan
// in the cache takes the next candidate of a learned search kept for its
// (device, operation, dtype, n, batch class), and two CUDA events are
// recorded around its launch on the caller's stream.  A later call of the
// same shape collects that time without waiting: if the events have not
// completed yet it simply runs the best plan seen so far.  When the search
// stops (stopping window or budget), its best plan goes into the plan cache,
// so every later call -- and bplg_query_plan -- uses it.  Every candidate is
// a valid plan, so results are exact throughout; only the speed varies while
// the search runs.  One candidate is in flight per shape at a time.
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "online.h"

namespace bplg {

int device_space(int op, int dtype, int64_t n, std::vector<bplg_plan> *plans, std::vector<int> *regs,
                 std::vector<int> *smem);

namespace {

struct OnlineState {
    std::vector<bplg_plan> plans;
    BoSearch *bo = nullptr;
    int pending = -1;       // candidate whose time is being measured
    bool recorded = false;  // its events were recorded (the launch succeeded)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool finished = false;
    ~OnlineState() {
        if (bo) bo_destroy(bo);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

using Key = std::tuple<int, int, int, int64_t, int>;  // device, op, dtype, n, batch class
std::mutex g_mu;
bool g_enabled = false;
int g_budget = 40;
uint64_t g_seed = 0;
std::map<Key, std::unique_ptr<OnlineState>> g_states;

int batch_class(int64_t batch) { return ilog2(batch < 1 ? 1 : batch); }

// fold a completed measurement into the search (lock held)
void collect(OnlineState &st) {
    if (st.pending < 0 || !st.recorded) return;
    const cudaError_t q = cudaEventQuery(st.e1);
    if (q == cudaErrorNotReady) return;
    float ms = -1.f;
    if (q != cudaSuccess || cudaEventElapsedTime(&ms, st.e0, st.e1) != cudaSuccess) ms = -1.f;
    bo_tell(st.bo, st.pending, static_cast<double>(ms));
    st.pending = -1;
    st.recorded = false;
}

}  // namespace

int online_set(bool enable, int budget, uint64_t seed) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_enabled = enable;
    g_budget = budget > 0 ? budget : 40;
    g_seed = seed;
    return BPLG_OK;
}

int online_plan(int op, int dtype, int64_t n, int64_t batch, bplg_plan *out, OnlineTicket *t) {
    t->applies = false;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_enabled) return BPLG_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    const Key key(dev, op, dtype, n, batch_class(batch));
    auto &slot = g_states[key];
    if (!slot) {
        std::unique_ptr<OnlineState> st(new OnlineState());
        int rc = device_space(op, dtype, n, &st->plans, nullptr, nullptr);
        if (rc != BPLG_OK) return rc;
        if (st->plans.empty()) return BPLG_OK;  // the regular path reports the error
        if ((e = cudaEventCreate(&st->e0)) != cudaSuccess || (e = cudaEventCreate(&st->e1)) != cudaSuccess)
            return cuda_error(e, "online tuning events");
        st->bo = bo_create(st->plans, g_budget, g_seed);
        slot = std::move(st);
    }
    OnlineState &st = *slot;
    collect(st);
    if (!st.finished && st.pending < 0) {
        const int next = bo_next(st.bo);
        if (next >= 0) {
            st.pending = next;
            st.recorded = false;
            *out = st.plans[next];
            t->applies = true;
            t->state = &st;
            t->e0 = st.e0;
            t->e1 = st.e1;
            return BPLG_OK;
        }
        st.finished = true;
        const int b = bo_best(st.bo);
        if (b >= 0) cache_store(op, dtype, n, batch, st.plans[b]);
    }
    const int b = bo_best(st.bo);
    if (b >= 0) {  // a measurement in flight, or the search has finished
        *out = st.plans[b];
        t->applies = true;
    }
    return BPLG_OK;
}

void online_launched(const OnlineTicket &t, cudaStream_t s, int launch_rc) {
    if (!t.state || !t.e1) return;
    std::lock_guard<std::mutex> lock(g_mu);
    OnlineState &st = *static_cast<OnlineState *>(t.state);
    if (launch_rc == BPLG_OK && cudaEventRecord(t.e1, s) == cudaSuccess) {
        st.recorded = true;
    } else {  // the candidate could not run: an invalid plan for the search
        bo_tell(st.bo, st.pending, -1.0);
        st.pending = -1;
        st.recorded = false;
    }
}

int online_status(int op, int dtype, int64_t n, int64_t batch, int32_t *evaluations, int32_t *finished,
                  bplg_plan *best) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    auto it = g_states.find(Key(dev, op, dtype, n, batch_class(batch)));
    if (best) std::memset(best, 0, sizeof(*best));
    if (it == g_states.end() || !it->second) {
        *evaluations = 0;
        *finished = 0;
        return BPLG_OK;
    }
    OnlineState &st = *it->second;
    collect(st);
    if (!st.finished && st.pending < 0 && bo_next(st.bo) < 0) {
        st.finished = true;
        const int b = bo_best(st.bo);
        if (b >= 0) cache_store(op, dtype, n, batch, st.plans[b]);
    }
    *evaluations = bo_evaluations(st.bo);
    *finished = st.finished ? 1 : 0;
    const int b = bo_best(st.bo);
    if (best && b >= 0) *best = st.plans[b];
    return BPLG_OK;
}

}  // namespace bplg
