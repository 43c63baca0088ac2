// extern "C" entry points: argument validation, plan resolution, dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "online.h"

namespace bplg {
const char *last_error_cstr();
void occupancy(const bplg_arch &a, int w, int regs, int smem, int *w_sm, int *b_a);
int guideline_select(const bplg_arch &a, const bplg_candidate *c, int count, bool radix_tunable);
double phi(const double *e, int count);
void arch_preset_tx1(bplg_arch *a);
void arch_preset_gb300(bplg_arch *a);
int arch_query(int dev, bplg_arch *a);
int plan_resources(const bplg_plan &p, int dtype, int64_t n, int *regs, int *smem, int *threads);
int device_space(int op, int dtype, int64_t n, std::vector<bplg_plan> *plans, std::vector<int> *regs,
                 std::vector<int> *smem);
int tune_search(const std::vector<bplg_plan> &plans, const std::vector<int> &regs, const std::vector<int> &smem,
                const bplg_arch &arch, int method, int budget, uint64_t seed,
                const std::function<double(const bplg_plan &)> &cost, int *chosen, bplg_tune_report *rep,
                const std::vector<double> *model_times);
int tune_on_device(int op, int dtype, int64_t n, int64_t batch, int method, int budget, uint64_t seed,
                   bplg_plan *out, bplg_tune_report *rep);
double time_plan(const bplg_plan &p, int dtype, int64_t n, int64_t batch, int reps, void *in, void *out,
                 void *b, void *c, void *d, cudaStream_t s, double limit_s);
int max_log_for(int op);
int time_plan_owned(const bplg_plan &p, int dtype, int64_t n, int64_t batch, int reps, double *ms);
int fft_device_status(int *flag, bool reset);
int tridiag_device_status(int *flag, bool reset);
int fft_tc_device_status(int *flag, bool reset);
int fft_tc_gemm_device_status(int *flag, bool reset);

namespace {
std::mutex g_default_mu;
std::map<std::tuple<int, int, int, int64_t>, bplg_plan> g_default;  // (device, op, dtype, n)

// Blocks the launch of a caller's plan would need, from the plan alone (no
// device query): one block per spb problems, or for the two-kernel FFT the
// larger of its two grids.  Saturates at kMaxGridBlocks + 1.
int64_t plan_blocks(const bplg_plan &p, int64_t n, int64_t batch) {
    if (p.op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog) && p.n1_log > 0 && p.n1_log < 31) {
        // at least one block per signal in each kernel
        if (batch > kMaxGridBlocks) return kMaxGridBlocks + 1;
        const int64_t n1 = int64_t(1) << p.n1_log, n2 = n / n1;
        const int64_t cols = p.spb > 0 ? batch * std::max<int64_t>(1, n2 / p.spb) : 0;
        const int64_t rows = p.row_spb > 0 ? batch * std::max<int64_t>(1, n1 / p.row_spb) : 0;
        return std::max(cols, rows);
    }
    return p.spb > 0 ? batch / p.spb + (batch % p.spb != 0 ? 1 : 0) : 0;
}

int resolve_plan(int op, int dtype, int64_t n, int64_t batch, const bplg_plan *given, bplg_plan *out,
                 OnlineTicket *ticket = nullptr) {
    if (given) {
        bplg_plan p = *given;
        if (p.op != op) return set_error(BPLG_ERR_INVALID_PLAN, "plan is for another operation");
        if (p.spb >= 1 && plan_blocks(p, n, batch) > kMaxGridBlocks) return check_grid(plan_blocks(p, n, batch), "plan");
        std::string why;
        int rc = check_plan_on_device(p, dtype, n, &why);
        if (rc == BPLG_ERR_INVALID_PLAN) return set_error(rc, "invalid plan: " + why);
        if (rc != BPLG_OK) return rc;
        *out = p;
        return BPLG_OK;
    }
    if (cache_lookup(op, dtype, n, batch, out)) return BPLG_OK;
    if (ticket) {
        const int rc = online_plan(op, dtype, n, batch, out, ticket);
        if (rc != BPLG_OK) return rc;
        if (ticket->applies) return BPLG_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    {
        std::lock_guard<std::mutex> lock(g_default_mu);
        auto it = g_default.find(std::make_tuple(dev, op, dtype, n));
        if (it != g_default.end()) {
            *out = it->second;
            return BPLG_OK;
        }
    }
    int rc = analytic_plan(op, dtype, n, out);
    if (rc != BPLG_OK) return rc;
    std::lock_guard<std::mutex> lock(g_default_mu);
    g_default[std::make_tuple(dev, op, dtype, n)] = *out;
    return BPLG_OK;
}

bool size_ok(int op, int64_t n, int64_t min_n) {
    return is_pow2(n) && n >= min_n && n <= (int64_t(1) << max_log_for(op));
}

bool overlaps(const void *p, size_t pn, const void *q, size_t qn) {
    const char *a = static_cast<const char *>(p);
    const char *b = static_cast<const char *>(q);
    return a < b + qn && b < a + pn;
}
}  // namespace
}  // namespace bplg

using namespace bplg;

extern "C" {

int bplg_scan_batched(int32_t dtype, const void *in, void *out, int64_t n, int64_t batch, const bplg_plan *plan,
                      void *stream) {
    clear_error();
    if (dtype != BPLG_I32 && dtype != BPLG_F32) return set_error(BPLG_ERR_INVALID_ARG, "scan: dtype must be I32 or F32");
    if (!in || !out) return set_error(BPLG_ERR_INVALID_ARG, "scan: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "scan: n and batch must be >= 1");
    if (n > (int64_t(1) << kScanMaxLog)) return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "scan: n must be <= 32768");
    if (!aligned16(in) || !aligned16(out)) return set_error(BPLG_ERR_INVALID_ARG, "scan: buffers must be 16-byte aligned");
    // any other n runs the plan of the next power of two, padded with zeros
    const int64_t np = next_pow2(n);
    bplg_plan p;
    OnlineTicket tk;
    int rc = resolve_plan(BPLG_OP_SCAN, dtype, np, batch, plan, &p, np == n ? &tk : nullptr);
    if (rc != BPLG_OK) return rc;
    p.n = static_cast<int32_t>(np);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tk.e0) cudaEventRecord(tk.e0, s);
    rc = scan_launch(p, dtype, in, out, n, batch, s);
    online_launched(tk, s, rc);
    return rc;
}

int bplg_fft_batched(const void *in, void *out, int64_t n, int64_t batch, int32_t dir, const bplg_plan *plan,
                     void *stream) {
    clear_error();
    if (!in || !out) return set_error(BPLG_ERR_INVALID_ARG, "fft: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "fft: n and batch must be >= 1");
    if (dir != -1 && dir != 1) return set_error(BPLG_ERR_INVALID_ARG, "fft: dir must be -1 or +1");
    if (!aligned16(in) || !aligned16(out)) return set_error(BPLG_ERR_INVALID_ARG, "fft: buffers must be 16-byte aligned");
    if (!is_pow2(n) && !plan && fft_mixed_supported(n))
        return fft_mixed_launch(in, out, n, batch, dir, static_cast<cudaStream_t>(stream));
    if (!is_pow2(n) && n > 2 && n <= (int64_t(1) << kBluesteinMaxLog))
        return fft_bluestein_launch(plan, in, out, n, batch, dir, static_cast<cudaStream_t>(stream));
    if (!size_ok(BPLG_OP_FFT, n, 2))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft: n must be in [2, 2^24] (at most 2^23 if not a power of two)");
    bplg_plan p;
    OnlineTicket tk;
    int rc = resolve_plan(BPLG_OP_FFT, BPLG_F32, n, batch, plan, &p, &tk);
    if (rc != BPLG_OK) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tk.e0) cudaEventRecord(tk.e0, s);
    rc = fft_launch(p, in, out, n, batch, dir, s);
    online_launched(tk, s, rc);
    return rc;
}

int bplg_fft_tc_batched(const void *in, void *out, int64_t n, int64_t batch, int32_t dir, int32_t precision,
                        const bplg_plan *plan, void *stream) {
    clear_error();
    if (!in || !out) return set_error(BPLG_ERR_INVALID_ARG, "fft tc: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "fft tc: n and batch must be >= 1");
    if (dir != -1 && dir != 1) return set_error(BPLG_ERR_INVALID_ARG, "fft tc: dir must be -1 or +1");
    if (precision != BPLG_TC_BF16 && precision != BPLG_TC_F16)
        return set_error(BPLG_ERR_INVALID_ARG, "fft tc: precision must be BPLG_TC_BF16 or BPLG_TC_F16");
    if (!size_ok(BPLG_OP_FFT_TC, n, 512))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft tc: n must be a power of two in [512, 16384]");
    if (!aligned16(in) || !aligned16(out)) return set_error(BPLG_ERR_INVALID_ARG, "fft tc: buffers must be 16-byte aligned");
    bplg_plan p;
    OnlineTicket tk;
    int rc = resolve_plan(BPLG_OP_FFT_TC, BPLG_F32, n, batch, plan, &p, &tk);
    if (rc != BPLG_OK) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tk.e0) cudaEventRecord(tk.e0, s);
    rc = fft_tc_launch(p, in, out, n, batch, dir, precision, s);
    online_launched(tk, s, rc);
    return rc;
}

int bplg_tridiag_batched(const float *a, const float *b, const float *c, const float *d, float *x, int64_t n,
                         int64_t batch, const bplg_plan *plan, void *stream) {
    clear_error();
    if (!a || !b || !c || !d || !x) return set_error(BPLG_ERR_INVALID_ARG, "tridiag: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "tridiag: n and batch must be >= 1");
    if (n < 2 || n > (int64_t(1) << kTridiagMaxLog))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "tridiag: n must be in [2, 8192]");
    for (const void *q : {(const void *)a, (const void *)b, (const void *)c, (const void *)d, (const void *)x})
        if (!aligned16(q)) return set_error(BPLG_ERR_INVALID_ARG, "tridiag: buffers must be 16-byte aligned");
    // the plan's op picks the solver: CR/PCR hybrid (default) or Wang-Mou;
    // any other n than a power of two runs Wang-Mou on the next power of two
    const int64_t np = next_pow2(n);
    if (np != n && plan && plan->op != BPLG_OP_TRIDIAG_WM)
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE,
                         "tridiag: n that is not a power of two needs a BPLG_OP_TRIDIAG_WM plan (or NULL)");
    const int op = np != n || (plan && plan->op == BPLG_OP_TRIDIAG_WM) ? BPLG_OP_TRIDIAG_WM : BPLG_OP_TRIDIAG;
    bplg_plan p;
    OnlineTicket tk;
    int rc = resolve_plan(op, BPLG_F32, np, batch, plan, &p, np == n ? &tk : nullptr);
    if (rc != BPLG_OK) return rc;
    p.n = static_cast<int32_t>(np);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tk.e0) cudaEventRecord(tk.e0, s);
    rc = op == BPLG_OP_TRIDIAG_WM ? tridiag_wm_launch(p, a, b, c, d, x, n, batch, s)
                                  : tridiag_launch(p, a, b, c, d, x, n, batch, s);
    online_launched(tk, s, rc);
    return rc;
}

int bplg_tridiag_refined(const float *a, const float *b, const float *c, const float *d, double *x, int64_t n,
                         int64_t batch, int32_t max_iter, double tol, int32_t *iters, const bplg_plan *plan,
                         void *stream) {
    clear_error();
    if (!a || !b || !c || !d || !x) return set_error(BPLG_ERR_INVALID_ARG, "refined: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "refined: n and batch must be >= 1");
    if (max_iter < 0 || max_iter > 64) return set_error(BPLG_ERR_INVALID_ARG, "refined: max_iter must be in [0, 64]");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return set_error(BPLG_ERR_INVALID_ARG, "refined: tol must be finite and >= 0");
    if (!size_ok(BPLG_OP_TRIDIAG_REFINED, n, 2))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "refined: n must be a power of two in [2, 4096]");
    for (const void *q : {(const void *)a, (const void *)b, (const void *)c, (const void *)d, (const void *)x})
        if (!aligned16(q)) return set_error(BPLG_ERR_INVALID_ARG, "refined: buffers must be 16-byte aligned");
    const size_t total = static_cast<size_t>(n) * static_cast<size_t>(batch);
    for (const void *q : {(const void *)a, (const void *)b, (const void *)c, (const void *)d})
        if (overlaps(x, total * 8, q, total * 4)) return set_error(BPLG_ERR_INVALID_ARG, "refined: x must not alias the inputs");
    bplg_plan p;
    OnlineTicket tk;
    int rc = resolve_plan(BPLG_OP_TRIDIAG_REFINED, BPLG_F32, n, batch, plan, &p, &tk);
    if (rc != BPLG_OK) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tk.e0) cudaEventRecord(tk.e0, s);
    rc = tridiag_refined_launch(p, a, b, c, d, x, n, batch, max_iter, tol, iters, s);
    online_launched(tk, s, rc);
    return rc;
}

int bplg_arch_query(int32_t device, bplg_arch *out) {
    clear_error();
    if (!out) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    return arch_query(device, out);
}

int bplg_arch_preset(int32_t which, bplg_arch *out) {
    clear_error();
    if (!out) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    if (which == 0) {
        arch_preset_tx1(out);
        return BPLG_OK;
    }
    if (which == 1) {
        arch_preset_gb300(out);
        return BPLG_OK;
    }
    return set_error(BPLG_ERR_INVALID_ARG, "unknown preset");
}

int bplg_occupancy(const bplg_arch *arch, int32_t warps_per_block, int32_t regs_per_thread, int32_t smem_per_block,
                   int32_t *w_sm, int32_t *b_a) {
    clear_error();
    if (!arch || !w_sm || !b_a) return set_error(BPLG_ERR_INVALID_ARG, "null argument");
    int w = 0, b = 0;
    occupancy(*arch, warps_per_block, regs_per_thread, smem_per_block, &w, &b);
    *w_sm = w;
    *b_a = b;
    return BPLG_OK;
}

int bplg_guideline_select(const bplg_arch *arch, const bplg_candidate *cands, int32_t count, int32_t radix_tunable,
                          int32_t *chosen) {
    clear_error();
    if (!arch || !chosen || count < 0 || (count > 0 && !cands)) return set_error(BPLG_ERR_INVALID_ARG, "bad argument");
    *chosen = count > 0 ? guideline_select(*arch, cands, count, radix_tunable != 0) : -1;
    return BPLG_OK;
}

double bplg_phi(const double *efficiencies, int32_t count) {
    if (!efficiencies) return 0.0;
    return phi(efficiencies, count);
}

int bplg_enumerate_plans(int32_t op, int32_t dtype, int64_t n, bplg_plan *out, int32_t capacity, int32_t *count) {
    clear_error();
    if (!count || capacity < 0 || (capacity > 0 && !out)) return set_error(BPLG_ERR_INVALID_ARG, "bad argument");
    if (max_log_for(op) < 0) return set_error(BPLG_ERR_INVALID_ARG, "unknown op");
    if (!size_ok(op, n, 1)) return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "unsupported size");
    std::vector<bplg_plan> plans;
    int rc = device_space(op, dtype, n, &plans, nullptr, nullptr);
    if (rc != BPLG_OK) return rc;
    *count = static_cast<int32_t>(plans.size());
    for (int i = 0; i < capacity && i < static_cast<int>(plans.size()); ++i) out[i] = plans[i];
    return BPLG_OK;
}

int bplg_plan_resources(const bplg_plan *plan, int32_t dtype, int32_t *regs, int32_t *smem, int32_t *threads) {
    clear_error();
    if (!plan || !regs || !smem || !threads) return set_error(BPLG_ERR_INVALID_ARG, "null argument");
    int r = 0, s = 0, t = 0;
    int rc = plan_resources(*plan, dtype, plan->n, &r, &s, &t);
    if (rc != BPLG_OK) return rc;
    *regs = r;
    *smem = s;
    *threads = t;
    return BPLG_OK;
}

int bplg_tune_plan(int32_t op, int32_t dtype, int64_t n, int64_t batch, int32_t method, int32_t budget, uint64_t seed,
                   bplg_plan *out, bplg_tune_report *report) {
    clear_error();
    if (!out) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    if (max_log_for(op) < 0) return set_error(BPLG_ERR_INVALID_ARG, "unknown op");
    if (batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "batch must be >= 1");
    if (method < BPLG_TUNE_ANALYTIC || method > BPLG_TUNE_MODEL) return set_error(BPLG_ERR_INVALID_ARG, "unknown method");
    if (!size_ok(op, n, op == BPLG_OP_SCAN ? 1 : (op == BPLG_OP_FFT_TC ? 512 : 2)))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "unsupported size");
    return tune_on_device(op, dtype, n, batch, method, budget, seed, out, report);
}

int bplg_tune_plans_cost(const bplg_plan *plans, int32_t count, const int32_t *regs, const int32_t *smem,
                         const bplg_arch *arch, int32_t method, int32_t budget, uint64_t seed, bplg_cost_fn cost,
                         void *user, int32_t *chosen, bplg_tune_report *report) {
    clear_error();
    if (!plans || count <= 0 || !chosen) return set_error(BPLG_ERR_INVALID_ARG, "bad argument");
    if (method < BPLG_TUNE_ANALYTIC || method > BPLG_TUNE_MODEL) return set_error(BPLG_ERR_INVALID_ARG, "unknown method");
    const bool analytical = method == BPLG_TUNE_ANALYTIC || method == BPLG_TUNE_MODEL;
    if (!analytical && !cost) return set_error(BPLG_ERR_INVALID_ARG, "a cost function is required");
    if (analytical && !arch) return set_error(BPLG_ERR_INVALID_ARG, "the analytical methods need arch limits");
    std::vector<bplg_plan> pv(plans, plans + count);
    std::vector<int> rv, sv;
    if (regs) rv.assign(regs, regs + count);
    if (smem) sv.assign(smem, smem + count);
    bplg_arch a;
    if (arch)
        a = *arch;
    else
        arch_preset_gb300(&a);
    std::vector<double> mt;
    if (method == BPLG_TUNE_MODEL) {
        const DevModel dm = dev_model_from_arch(a, 0.0, 0.0);
        const int64_t n = plans[0].n > 0 ? plans[0].n : 1;
        const int64_t batch = std::max<int64_t>(1, (int64_t(1) << 24) / n);
        for (int i = 0; i < count; ++i)
            mt.push_back(model_plan_time(pv[i], n, batch, rv.empty() ? 32 : rv[i], sv.empty() ? 0 : sv[i], 0, 0, dm));
    }
    int ch = -1;
    int rc = tune_search(pv, rv, sv, a, method, budget, seed,
                         [&](const bplg_plan &p) { return cost ? cost(&p, user) : NAN; }, &ch, report, &mt);
    *chosen = ch;
    return rc;
}

int bplg_query_plan(int32_t op, int32_t dtype, int64_t n, int64_t batch, bplg_plan *out) {
    clear_error();
    if (!out) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    if (max_log_for(op) < 0) return set_error(BPLG_ERR_INVALID_ARG, "unknown op");
    if (batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "batch must be >= 1");
    if (!size_ok(op, n, op == BPLG_OP_SCAN ? 1 : (op == BPLG_OP_FFT_TC ? 512 : 2)))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "unsupported size");
    return resolve_plan(op, dtype, n, batch, nullptr, out);
}

int bplg_check_plan(const bplg_plan *plan, int32_t dtype, int64_t n) {
    clear_error();
    if (!plan) return set_error(BPLG_ERR_INVALID_ARG, "null plan");
    std::string why;
    int rc = check_plan_on_device(*plan, dtype, n, &why);
    if (rc == BPLG_ERR_INVALID_PLAN) return set_error(rc, "invalid plan: " + why);
    return rc;
}

int bplg_time_plan(const bplg_plan *plan, int32_t dtype, int64_t n, int64_t batch, int32_t reps, double *median_ms) {
    clear_error();
    if (!plan || !median_ms || reps < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "bad argument");
    std::string why;
    int rc = check_plan_on_device(*plan, dtype, n, &why);
    if (rc == BPLG_ERR_INVALID_PLAN) return set_error(rc, "invalid plan: " + why);
    if (rc != BPLG_OK) return rc;
    return time_plan_owned(*plan, dtype, n, batch, reps, median_ms);
}

int bplg_set_online_tuning(int32_t enable, int32_t budget, uint64_t seed) {
    clear_error();
    if (budget < 0) return set_error(BPLG_ERR_INVALID_ARG, "budget must be >= 0");
    return online_set(enable != 0, budget, seed);
}

int bplg_online_status(int32_t op, int32_t dtype, int64_t n, int64_t batch, int32_t *evaluations,
                       int32_t *finished, bplg_plan *best) {
    clear_error();
    if (!evaluations || !finished) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    if (max_log_for(op) < 0) return set_error(BPLG_ERR_INVALID_ARG, "unknown op");
    return online_status(op, dtype, n, batch, evaluations, finished, best);
}

int bplg_device_status(int32_t *flag, int32_t reset) {
    clear_error();
    if (!flag) return set_error(BPLG_ERR_INVALID_ARG, "null output");
    int f1 = 0, f2 = 0, f3 = 0, f4 = 0;
    int rc = fft_device_status(&f1, reset != 0);
    if (rc != BPLG_OK) return rc;
    rc = tridiag_device_status(&f2, reset != 0);
    if (rc != BPLG_OK) return rc;
    rc = fft_tc_device_status(&f3, reset != 0);
    if (rc != BPLG_OK) return rc;
    rc = fft_tc_gemm_device_status(&f4, reset != 0);
    if (rc != BPLG_OK) return rc;
    *flag = f1 ? f1 : (f2 ? f2 : (f3 ? f3 : f4));
    return BPLG_OK;
}

const char *bplg_last_error(void) { return last_error_cstr(); }

int32_t bplg_version(void) { return 100; }

}  // extern "C"
