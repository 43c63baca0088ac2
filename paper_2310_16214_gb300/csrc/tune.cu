// Tuning (Section IV): the occupancy relations and analytical guideline of
// Section IV-A, the Bayesian-optimisation search of Section IV-B with a
// Gaussian-process cost model and expected improvement, exhaustive search,
// the Phi metric of Section VI, and the GPU timing of one candidate (the
// objective f(a_j, x_B) = execution time).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.h"

namespace bplg {

// ---------------------------------------------------------------- occupancy
static int ceil_to(int x, int unit) { return unit > 0 ? ((x + unit - 1) / unit) * unit : x; }

void occupancy(const bplg_arch &a, int w, int regs, int smem, int *w_sm, int *b_a) {
    *w_sm = 0;
    *b_a = 0;
    if (w <= 0 || w * 32 > a.max_threads_per_block || regs > a.max_regs_per_thread || smem > a.max_smem_per_block)
        return;
    int by_warps = a.max_warps_per_sm / w;
    int by_regs = a.max_blocks_per_sm;
    if (regs > 0) {
        int per_warp = ceil_to(regs * 32, a.reg_alloc_unit);
        int warps = a.regs_per_sm / per_warp;
        if (a.warp_alloc_granularity > 0) warps -= warps % a.warp_alloc_granularity;
        by_regs = warps / w;
    }
    int by_smem = a.max_blocks_per_sm;
    int need = smem + a.smem_reserved_per_block;
    if (need > 0) by_smem = a.smem_per_sm / ceil_to(need, a.smem_alloc_unit);
    int b = std::min(std::min(a.max_blocks_per_sm, by_warps), std::min(by_regs, by_smem));
    if (b < 0) b = 0;
    *b_a = b;
    *w_sm = b * w;
}

// ------------------------------------------------------- analytical guideline
// Section IV-A, read as: (premise i) prefer shuffle communication when some
// shuffle candidate keeps >= 60 % warp occupancy; (bullet 4) for radix-tunable
// algorithms keep the largest radix among candidates with >= 60 % warp
// occupancy; then (bullet 1) W_SM = W^max and B_a = B^max -> largest P;
// (bullet 2) W_SM / W^max in [60 %, 100 %] -> largest B_a, then largest P;
// (bullet 3) otherwise largest W_SM, then largest P, then largest B_a.
// Full ties keep the earliest candidate.
int guideline_select(const bplg_arch &a, const bplg_candidate *c, int count, bool radix_tunable) {
    std::vector<int> w(count), b(count), pool;
    for (int i = 0; i < count; ++i) {
        occupancy(a, (c[i].L + 31) / 32, c[i].regs, c[i].smem, &w[i], &b[i]);
        if (b[i] > 0) pool.push_back(i);
    }
    if (pool.empty()) return -1;
    const double wmax = a.max_warps_per_sm;
    auto ratio = [&](int i) { return w[i] / wmax; };
    bool shuf_ok = false;
    for (int i : pool)
        if (c[i].shuffle && ratio(i) >= 0.6) shuf_ok = true;
    if (shuf_ok) {
        std::vector<int> p2;
        for (int i : pool)
            if (c[i].shuffle) p2.push_back(i);
        pool.swap(p2);
    }
    if (radix_tunable) {
        int rmax = -1;
        for (int i : pool)
            if (ratio(i) >= 0.6) rmax = std::max(rmax, c[i].radix);
        if (rmax > 0) {
            std::vector<int> p2;
            for (int i : pool)
                if (c[i].radix == rmax) p2.push_back(i);
            pool.swap(p2);
        }
    }
    int best = -1;
    // bullet 1
    for (int i : pool)
        if (w[i] == a.max_warps_per_sm && b[i] == a.max_blocks_per_sm)
            if (best < 0 || c[i].P > c[best].P) best = i;
    if (best >= 0) return best;
    // bullet 2
    for (int i : pool) {
        if (ratio(i) < 0.6 || ratio(i) > 1.0) continue;
        if (best < 0 || b[i] > b[best] || (b[i] == b[best] && c[i].P > c[best].P)) best = i;
    }
    if (best >= 0) return best;
    // bullet 3
    for (int i : pool) {
        if (best < 0 || w[i] > w[best] || (w[i] == w[best] && c[i].P > c[best].P) ||
            (w[i] == w[best] && c[i].P == c[best].P && b[i] > b[best]))
            best = i;
    }
    return best;
}

double phi(const double *e, int count) {
    if (count <= 0) return 0.0;
    double s = 0.0;
    for (int i = 0; i < count; ++i) {
        if (!(e[i] > 0.0)) return 0.0;
        s += 1.0 / e[i];
    }
    return count / s;
}

// ------------------------------------------------------------- arch limits
void arch_preset_tx1(bplg_arch *a) {
    *a = bplg_arch{64, 32, 65536, 256, 4, 255, 65536, 256, 49152, 0, 1024, 2};
}
void arch_preset_gb300(bplg_arch *a) {
    *a = bplg_arch{64, 32, 65536, 256, 4, 255, 233472, 128, 232448, 1024, 1024, 152};
}

int arch_query(int dev, bplg_arch *a) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return set_error(BPLG_ERR_NO_DEVICE, "no CUDA device");
    if (dev < 0 || dev >= count) return set_error(BPLG_ERR_INVALID_ARG, "device index out of range");
    cudaDeviceProp p;
    e = cudaGetDeviceProperties(&p, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
    a->max_warps_per_sm = p.maxThreadsPerMultiProcessor / 32;
    a->max_blocks_per_sm = p.maxBlocksPerMultiProcessor;
    a->regs_per_sm = p.regsPerMultiprocessor;
    a->reg_alloc_unit = 256;
    a->warp_alloc_granularity = 4;
    a->max_regs_per_thread = 255;
    a->smem_per_sm = static_cast<int32_t>(p.sharedMemPerMultiprocessor);
    a->smem_alloc_unit = 128;
    a->max_smem_per_block = static_cast<int32_t>(p.sharedMemPerBlockOptin);
    a->smem_reserved_per_block = static_cast<int32_t>(p.reservedSharedMemPerBlock);
    a->max_threads_per_block = p.maxThreadsPerBlock;
    a->num_sms = p.multiProcessorCount;
    return BPLG_OK;
}

// ------------------------------------------------------ candidates on device
bool launch_info_for(const bplg_plan &p, int dtype, int64_t n, Launch *li);

namespace {
std::mutex g_fa_mu;
std::map<std::pair<int, const void *>, cudaFuncAttributes> g_fa;

int func_attrs(const void *f, cudaFuncAttributes *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_fa_mu);
    auto key = std::make_pair(dev, f);
    auto it = g_fa.find(key);
    if (it != g_fa.end()) {
        *out = it->second;
        return BPLG_OK;
    }
    e = cudaFuncGetAttributes(out, f);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes");
    g_fa[key] = *out;
    return BPLG_OK;
}
}  // namespace

int plan_resources(const bplg_plan &p, int dtype, int64_t n, int *regs, int *smem, int *threads) {
    Launch li;
    if (!launch_info_for(p, dtype, n, &li)) return set_error(BPLG_ERR_INVALID_PLAN, "plan has no kernel");
    cudaFuncAttributes fa;
    int rc = func_attrs(li.func, &fa);
    if (rc != BPLG_OK) return rc;
    *regs = fa.numRegs;
    *smem = li.smem + static_cast<int>(fa.sharedSizeBytes);
    *threads = li.threads;
    return BPLG_OK;
}

// valid plans on the current device with their resources
int device_space(int op, int dtype, int64_t n, std::vector<bplg_plan> *plans, std::vector<int> *regs,
                 std::vector<int> *smem) {
    std::vector<bplg_plan> all = enumerate_structural(op, dtype, n);
    for (const auto &p : all) {
        std::string why;
        int rc = check_plan_on_device(p, dtype, n, &why);
        if (rc == BPLG_ERR_INVALID_PLAN) continue;
        if (rc != BPLG_OK) return rc;
        int r = 0, s = 0, t = 0;
        rc = plan_resources(p, dtype, n, &r, &s, &t);
        if (rc != BPLG_OK) return rc;
        plans->push_back(p);
        if (regs) regs->push_back(r);
        if (smem) smem->push_back(s);
    }
    return BPLG_OK;
}

static bplg_candidate to_candidate(const bplg_plan &p, int regs, int smem) {
    bplg_candidate c;
    std::memset(&c, 0, sizeof(c));
    c.S = p.S;
    c.P = p.P;
    c.L = p.L;
    c.regs = regs;
    c.smem = smem;
    c.radix = p.radix;
    c.shuffle = p.op == BPLG_OP_SCAN ? 0 : p.shuffle;  // scan always shuffles: no preference signal
    return c;
}

// model time of every plan of a device space (the two-kernel FFT's row
// kernel resources looked up here)
int model_times_on_device(int dev, const std::vector<bplg_plan> &plans, const std::vector<int> &regs,
                          const std::vector<int> &smem, int64_t n, int64_t batch, std::vector<double> *out) {
    DevModel dm;
    int rc = dev_model_query(dev, &dm);
    if (rc != BPLG_OK) return rc;
    out->assign(plans.size(), INFINITY);
    for (size_t i = 0; i < plans.size(); ++i) {
        int r2 = 0, s2 = 0;
        if (plans[i].op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog)) {
            Launch l2;
            if (!fft_large_launch_info(plans[i], n, 1, -1, 1, &l2)) continue;
            cudaFuncAttributes fa;
            rc = func_attrs(l2.func, &fa);
            if (rc != BPLG_OK) return rc;
            r2 = fa.numRegs;
            s2 = l2.smem + static_cast<int>(fa.sharedSizeBytes);
        }
        (*out)[i] = model_plan_time(plans[i], n, batch, regs[i], smem[i], r2, s2, dm);
    }
    return BPLG_OK;
}

// The default plan of a plan-less call: the GB300 cost model's choice for a
// batch of 2^24 / n problems (or one problem above that size).
int analytic_plan(int op, int dtype, int64_t n, bplg_plan *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::vector<bplg_plan> plans;
    std::vector<int> regs, smem;
    int rc = device_space(op, dtype, n, &plans, &regs, &smem);
    if (rc != BPLG_OK) return rc;
    if (plans.empty()) return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "no valid plan for this size");
    const int64_t batch = std::max<int64_t>(1, (int64_t(1) << 24) / n);
    std::vector<double> t;
    rc = model_times_on_device(dev, plans, regs, smem, n, batch, &t);
    if (rc != BPLG_OK) return rc;
    int k = -1;
    for (size_t i = 0; i < plans.size(); ++i)
        if (std::isfinite(t[i]) && (k < 0 || t[i] < t[k])) k = static_cast<int>(i);
    if (k < 0) return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "no plan can launch");
    *out = plans[k];
    return BPLG_OK;
}

// ------------------------------------------------ GB300 analytical cost model
// A zero-evaluation estimate of a plan's time on the current device, built
// from the premises of Section IV-A restated for this GPU: coalescing (the
// 128-byte lines a warp-wide global access touches), occupancy (resident
// blocks from the kernel's real register and shared-memory counts), the
// latency that resident work must hide (Little's law: B_a blocks in flight,
// each living one HBM round trip plus its own transfer and compute time),
// the instruction issue rate, barriers per stage, the block launch rate,
// and, for the refined solve, the FP64 pipe.  The terms combine as a soft
// maximum (an L4 norm), so the bound that dominates decides and the others
// break ties.  Per-op instruction counts per thread follow the kernels'
// algorithms (radix-r butterflies and exchanges per Stockham stage, CR
// levels in registers or shared memory, Wang-Mou merge stages, the two
// residuals and two solves of one refinement).  The constants are properties
// of the device class, fixed once:
//   latency          0.75 us  loaded HBM round trip of a block's first loads
//   cpi              6        clocks per dependent instruction of one warp
//   barrier          40       clocks per block barrier, x (1 + warps / 16)
//   block launch     80 ns    per block per SM (launch and retire)
//   issue            4        warp instructions per clock per SM
//   line             1        clock per 128-byte line of a warp-wide access
//   FP64             2        fused multiply-adds per clock per SM
//   clock, bandwidth 0.92 x the peak SM clock, 0.83 x the nominal HBM rate
//                    (what sustained streaming reaches)
// A pipelined plan (bulk-copy ring) hides half the latency.
namespace {

constexpr double kModelLatency = 0.75e-6;
constexpr double kModelCpi = 6.0;
constexpr double kModelBarrier = 40.0;
constexpr double kModelBlockLaunch = 80e-9;
constexpr double kModelIpc = 4.0;
constexpr double kModelLine = 1.0;
constexpr double kModelFp64PerClk = 2.0;
constexpr double kModelNorm = 4.0;

struct ModelOp {
    double instr = 0;   // instructions per thread
    double bars = 0;    // block barriers
    double bpe = 0;     // algorithmic HBM bytes per element
    double acc = 0;     // warp-wide global access instructions per thread
    double lines = 1;   // 128-byte lines per such access
    bool piped = false; // bulk-copy ring in front of the loads
    bool persistent = false;  // one block per SM looping over tiles, the next tile's loads in flight
    double fp64 = 0;    // FP64 pipe operations per element
};

int lg2i(int64_t v) { return ilog2(v < 1 ? 1 : v); }

// lines of one warp-wide access when consecutive threads are `stride` bytes
// apart and each moves `bytes`
double warp_lines(double stride, double bytes) {
    if (stride <= bytes) return std::max(1.0, std::ceil(32.0 * bytes / 128.0));
    return std::min(32.0, std::max(1.0, std::ceil(32.0 * stride / 128.0)));
}

// lines of a warp-wide access over 32 threads in groups of g contiguous
// `bytes`-wide elements, the groups far apart
double grouped_lines(int64_t g, double bytes) {
    if (g >= 32) return std::max(1.0, std::ceil(32.0 * bytes / 128.0));
    return static_cast<double>(32 / g) * std::max(1.0, std::ceil(g * bytes / 128.0));
}

ModelOp model_op(const bplg_plan &p, int64_t n) {
    ModelOp m;
    const int P = std::max(1, p.P);
    const int64_t tps = std::max<int64_t>(1, n / P);
    switch (p.op) {
        case BPLG_OP_SCAN:
            m.bpe = 8;
            m.instr = P * 2.0 + 14 + (tps > 32 ? 12 : 0);
            m.bars = tps > 32 ? 1 : 0;
            m.acc = 2.0 * std::max(1, P / 4);
            m.lines = warp_lines(P * 4.0, P >= 4 ? 16.0 : P * 4.0);
            break;
        case BPLG_OP_FFT:
        case BPLG_OP_FFT_TC: {
            m.bpe = 16;
            if (p.op == BPLG_OP_FFT_TC && p.io == 2) {
                // two 64-point GEMM passes in a persistent loop: per element
                // two splits and operand stores, one twiddle, two
                // tensor-memory reads with neighbour exchanges (about 60
                // instructions); the next tile's loads in flight behind the
                // products
                m.instr = P * 60.0 + 100;
                m.bars = 4;
                m.acc = 2.0 * P;
                m.lines = 2;
                m.persistent = true;
                break;
            }
            const int r = p.radix, lr = lg2i(r), logn = lg2i(n);
            const int K = (logn + lr - 1) / lr;
            const bool spec = p.smem_pad == 1 && ((p.io == 0 && ((r == 16 && logn >= 5 && logn <= 14) ||
                                                                  (r == 8 && logn >= 4 && logn <= 9))) ||
                                                  (p.io == 2 && r == 16 && logn >= 10 && logn <= 14));
            const double bf = r == 2 ? 2.0 : r == 4 ? 3.0 : r == 8 ? 4.5 : 5.5;  // butterfly, per element
            double idx = spec ? 0.5 : 3.0;                                       // stage index arithmetic
            double xch = 2.0 * (K - 1) * (p.smem_pad ? 1.0 : 2.0);               // exchanges (bank conflicts unpadded)
            if (p.smem_layout == 1) xch *= 2;                                    // real and imaginary in turn
            double stage = bf + 3.0 + idx;                                       // + twiddle
            if (p.op == BPLG_OP_FFT_TC) stage += p.io == 0 ? 6.0 : 30.0;          // hi/lo split, MMA round trip
            m.instr = r * (K * stage + xch) + 12;
            // tensor-core stages: io 0 waits each stage for its tcgen05
            // products (write A, barrier, issue, commit, mbarrier wait,
            // tensor-memory read: two hand-offs, about 1 us a stage, 32
            // barriers' worth); io 1 gathers fragments
            m.bars = 2.0 * (K - 1) + (p.op == BPLG_OP_FFT_TC ? (p.io == 0 ? 32.0 : 2.0) * K : 0.0);
            if (p.io == 1) {
                m.instr += r * 4;
                m.bars += 2;
                m.acc = 2.0 * std::max(1, r / 2);
                m.lines = 4;
            } else if (p.io == 0) {
                m.acc = 2.0 * r;
                m.lines = std::max(2.0, grouped_lines(tps, 8.0));
            } else {
                m.acc = 2.0 * std::max(1, r / 2);
                m.lines = 4;
                m.piped = true;
            }
            break;
        }
        case BPLG_OP_TRIDIAG: {
            m.bpe = 20;
            const int64_t mm = std::max(1, p.cr_switch);
            const int lay = p.smem_layout;
            const int lvl = std::max(0, lg2i(n / mm) - (lay == 2 ? lg2i(P) : 0));
            const double per_eq = 20.0 * (p.smem_pad ? 1.0 : 2.0);
            const double eq_thread = (lay == 2 ? static_cast<double>(n) / P : static_cast<double>(n)) / tps;
            const bool shuf = p.shuffle && mm <= 32;
            m.instr = P * 10.0 + (lay == 2 ? lg2i(P) * P * 6.0 : 0.0) + lvl * per_eq * std::max(1.0, eq_thread) +
                      lg2i(mm) * (shuf ? 14.0 : 36.0) + 12;
            m.bars = 2.0 * lvl + (shuf ? 0.0 : 2.0 * lg2i(mm)) + 2;
            m.acc = 5.0 * std::max(1, P / 4);
            m.lines = warp_lines(P * 4.0, P >= 4 ? 16.0 : P * 4.0);
            m.piped = p.io == 1;
            break;
        }
        case BPLG_OP_TRIDIAG_WM: {
            m.bpe = 20;
            const int r = p.radix, lr = lg2i(r);
            const int st = tps > 1 ? (lg2i(tps) + lr - 1) / lr : 0;
            const double merge = r == 2 ? 45.0 : r == 4 ? 100.0 : 220.0;
            int smst = 0;
            for (int k = 0; k < st; ++k)
                if (!(p.shuffle && (k + 1) * lr <= 5)) ++smst;
            m.instr = P * 20.0 + st * merge + smst * 10.0 + 12;
            m.bars = 2.0 * smst + ((p.shuffle && tps <= 32) ? 0.0 : 1.0);
            m.acc = 5.0 * std::max(1, P / 4);
            m.lines = warp_lines(P * 4.0, P >= 4 ? 16.0 : P * 4.0);
            break;
        }
        case BPLG_OP_TRIDIAG_REFINED: {
            m.bpe = 24;
            const int lay = p.smem_layout;
            const double solve = lay == 7 ? P * 20.0 + lg2i(tps) * 45.0
                                          : P * 30.0 + 150.0 + (lay >= 4 ? 0.0 : static_cast<double>(n) / tps * 40.0);
            m.instr = 2 * solve + P * 70.0 + 100;
            m.bars = lay == 7 ? 16 : 60;
            m.acc = 6.0 * std::max(1, P / 4);
            m.lines = warp_lines(P * 4.0, P >= 4 ? 16.0 : P * 4.0);
            m.fp64 = 7;  // two residuals of 3 FMA and one update per element (one correction)
            break;
        }
        default:
            break;
    }
    return m;
}

// Time of one kernel: `blocks` blocks of `threads` threads over elems
// elements, with this kernel's registers and shared memory.
double model_kernel(const ModelOp &m, const DevModel &dm, int64_t elems, int64_t blocks, int threads, int regs,
                    int smem, int spb_elems) {
    int w_sm = 0, b_a = 0;
    occupancy(dm.arch, (threads + 31) / 32, regs, smem, &w_sm, &b_a);
    if (b_a <= 0) return INFINITY;
    const double sms = dm.arch.num_sms;
    const double wpb = (threads + 31) / 32;
    const double per_sm_blocks = static_cast<double>(blocks) / sms;
    const double bw_sm = dm.bw / sms;
    const double t_xfer = static_cast<double>(spb_elems) * m.bpe / bw_sm;
    const double t_comp = std::max(wpb * m.instr / kModelIpc, m.instr * kModelCpi) / dm.clk +
                          m.bars * kModelBarrier * (1.0 + wpb / 16.0) / dm.clk;
    const double res = kModelLatency * (m.piped ? 0.5 : 1.0) + t_xfer + t_comp;
    // a persistent block overlaps a tile's transfer with the previous tile's
    // work and pays the latency and the launch once
    const double t_lat = m.persistent ? per_sm_blocks * std::max(t_xfer, t_comp) / b_a + kModelLatency
                                      : per_sm_blocks * res / b_a;
    const double terms[6] = {
        t_lat,                                                            // latency, b_a blocks (tiles) in flight
        static_cast<double>(elems) * m.bpe / dm.bw,                       // HBM bandwidth
        per_sm_blocks * wpb * m.instr / (kModelIpc * dm.clk),             // issue
        per_sm_blocks * wpb * m.acc * m.lines * kModelLine / dm.clk,      // lines through the load/store unit
        (m.persistent ? 1.0 : per_sm_blocks) * kModelBlockLaunch,         // block launches
        static_cast<double>(elems) * m.fp64 / (sms * kModelFp64PerClk * dm.clk)};  // FP64 pipe
    double s = 0.0;
    for (double t : terms) s += std::pow(t, kModelNorm);
    return std::pow(s, 1.0 / kModelNorm);
}

}  // namespace

DevModel dev_model_from_arch(const bplg_arch &a, double peak_clock_hz, double nominal_bw) {
    DevModel d;
    d.arch = a;
    d.clk = 0.92 * (peak_clock_hz > 0 ? peak_clock_hz : 2.07e9);
    d.bw = 0.83 * (nominal_bw > 0 ? nominal_bw : 8.18e12);
    return d;
}

int dev_model_query(int dev, DevModel *out) {
    bplg_arch a;
    int rc = arch_query(dev, &a);
    if (rc != BPLG_OK) return rc;
    int clk_khz = 0, mem_khz = 0, bus_bits = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    cudaDeviceGetAttribute(&mem_khz, cudaDevAttrMemoryClockRate, dev);
    cudaDeviceGetAttribute(&bus_bits, cudaDevAttrGlobalMemoryBusWidth, dev);
    const double bw = 2.0 * mem_khz * 1e3 * bus_bits / 8.0;  // double data rate
    *out = dev_model_from_arch(a, clk_khz * 1e3, bw);
    return BPLG_OK;
}

// Modelled time (seconds) of plan p for (n, batch).  regs/smem are the
// kernel's resources; for the two-kernel FFT regs2/smem2 are those of the
// row kernel (the column kernel's are regs/smem).
double model_plan_time(const bplg_plan &p, int64_t n, int64_t batch, int regs, int smem, int regs2, int smem2,
                       const DevModel &dm) {
    if (p.op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog) && p.n1_log > 0) {
        const int l1 = p.n1_log, l2 = lg2i(n) - p.n1_log;
        const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
        // a pass whose HBM accesses are segments of `seg` contiguous bytes
        // (rows far apart) pays for partial lines: sqrt(128 / seg) per byte
        // below a whole 128-byte line (32 bytes cost twice as much)
        auto seg_cost = [](double seg) { return std::sqrt(std::max(1.0, 128.0 / seg)); };
        auto pass = [&](int64_t len, int per_block, int64_t cnt, int rg, int sm, double lines, double bytes_factor) {
            bplg_plan q = p;
            q.radix = q.P = 16;
            q.io = 0;
            q.smem_pad = 1;
            q.smem_layout = 0;
            ModelOp m = model_op(q, len);
            m.instr += 16 * 4.0;  // the large-transform twiddle or the transposed store
            m.lines = lines;
            m.bpe *= bytes_factor;
            const int threads = static_cast<int>(per_block * (len / 16));
            return model_kernel(m, dm, n * batch, batch * cnt, threads, rg, sm, static_cast<int>(per_block * len));
        };
        // columns: loads and stores in segments of spb values; rows: loads
        // whole rows, stores transposed in segments of row_spb values
        const double c = pass(n1, p.spb, n2 / std::max(1, p.spb), regs, smem, grouped_lines(p.spb, 8.0),
                              seg_cost(8.0 * p.spb));
        const double r = pass(n2, p.row_spb, n1 / std::max(1, p.row_spb), regs2 > 0 ? regs2 : regs,
                              smem2 > 0 ? smem2 : smem, grouped_lines(p.row_spb, 8.0),
                              0.5 * (1.0 + seg_cost(8.0 * p.row_spb)));
        return c + r;
    }
    const ModelOp m = model_op(p, n);
    const int64_t spb = std::max(1, p.spb);
    const int64_t blocks = (batch + spb - 1) / spb;  // tiles of a persistent kernel
    // the 4096-point two-pass tensor-core kernel adds the warp that issues the products
    const int threads = p.op == BPLG_OP_FFT_TC && p.io == 2 && n == 4096 ? p.L + 32 : p.L;
    return model_kernel(m, dm, n * batch, blocks, threads, regs, smem, static_cast<int>(spb * n));
}

// ------------------------------------------------- Bayesian optimisation
namespace {

struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// knob vector of a plan, before normalisation: log2 of the graded knobs, the
// binary knobs as 0/1, and the categorical knobs (shared-memory layout, io
// mode) one-hot, so that two layouts are equally far apart
std::vector<double> raw_features(const bplg_plan &p) {
    std::vector<double> f = {std::log2(double(p.P)), std::log2(double(p.spb)), double(p.pattern),
                             double(p.smem_pad), std::log2(double(std::max(1, p.cr_switch))), double(p.shuffle)};
    for (int k = 0; k < 8; ++k) f.push_back(p.smem_layout == k ? 1.0 : 0.0);
    for (int k = 0; k < 3; ++k) f.push_back(p.io == k ? 1.0 : 0.0);
    // the merge radix of the Wang-Mou solver (a constant column elsewhere,
    // dropped by the normalisation)
    f.push_back(p.op == BPLG_OP_TRIDIAG_WM ? std::log2(double(p.radix)) : 0.0);
    return f;
}

std::vector<std::vector<double>> encode(const std::vector<bplg_plan> &plans) {
    std::vector<std::vector<double>> raw;
    for (const auto &p : plans) raw.push_back(raw_features(p));
    const size_t d = raw.empty() ? 0 : raw[0].size();
    std::vector<double> lo(d, 1e300), hi(d, -1e300);
    for (const auto &r : raw)
        for (size_t k = 0; k < d; ++k) {
            lo[k] = std::min(lo[k], r[k]);
            hi[k] = std::max(hi[k], r[k]);
        }
    std::vector<std::vector<double>> out;
    for (const auto &r : raw) {
        std::vector<double> f;
        for (size_t k = 0; k < d; ++k)
            if (hi[k] > lo[k]) f.push_back((r[k] - lo[k]) / (hi[k] - lo[k]));
        out.push_back(f);
    }
    return out;
}

// Matern-5/2 covariance with one lengthscale per knob (ARD)
double matern52(const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &ell) {
    double s = 0.0;
    for (size_t k = 0; k < x.size(); ++k) {
        const double t = (x[k] - y[k]) / ell[k];
        s += t * t;
    }
    const double q = std::sqrt(5.0 * s);
    return (1.0 + q + q * q / 3.0) * std::exp(-q);
}

// in-place Cholesky of an n x n SPD matrix (lower); false if not SPD
bool cholesky(std::vector<double> &K, int n) {
    for (int j = 0; j < n; ++j) {
        double s = K[j * n + j];
        for (int k = 0; k < j; ++k) s -= K[j * n + k] * K[j * n + k];
        if (s <= 0.0) return false;
        const double l = std::sqrt(s);
        K[j * n + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double t = K[i * n + j];
            for (int k = 0; k < j; ++k) t -= K[i * n + k] * K[j * n + k];
            K[i * n + j] = t / l;
        }
    }
    return true;
}

void solve_lower(const std::vector<double> &L, int n, std::vector<double> &b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
        b[i] = s / L[i * n + i];
    }
}
void solve_upper_t(const std::vector<double> &L, int n, std::vector<double> &b) {
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * b[k];
        b[i] = s / L[i * n + i];
    }
}

struct GP {
    std::vector<std::vector<double>> X;
    std::vector<double> L, alpha, ell;
    double mean = 0.0, scale = 1.0;
    int n = 0;

    bool fit_with(const std::vector<std::vector<double>> &Xs, const std::vector<double> &ys,
                  const std::vector<double> &l, double noise, double *lml) {
        n = static_cast<int>(Xs.size());
        X = Xs;
        ell = l;
        L.assign(size_t(n) * n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j <= i; ++j) {
                double k = matern52(X[i], X[j], ell);
                if (i == j) k += noise;
                L[i * n + j] = k;
                L[j * n + i] = k;
            }
        if (!cholesky(L, n)) return false;
        alpha = ys;
        solve_lower(L, n, alpha);
        double quad = 0.0;
        for (double v : alpha) quad += v * v;
        solve_upper_t(L, n, alpha);
        double logdet = 0.0;
        for (int i = 0; i < n; ++i) logdet += std::log(L[i * n + i]);
        *lml = -0.5 * quad - logdet;
        return true;
    }

    // Prior mean = the worst observed log time (a pessimistic prior: an
    // unexplored plan is expected to be as slow as the slowest seen, so
    // expected improvement concentrates near good plans); prior scale = the
    // spread of the observations.  Lengthscales: coordinate-wise search over
    // a grid, two sweeps, maximising the log marginal likelihood.
    void fit(const std::vector<std::vector<double>> &Xs, const std::vector<double> &y) {
        const double avg = std::accumulate(y.begin(), y.end(), 0.0) / y.size();
        double var = 0.0;
        for (double v : y) var += (v - avg) * (v - avg);
        mean = *std::max_element(y.begin(), y.end());
        scale = std::sqrt(var / y.size());
        if (scale < 1e-9) scale = 1e-9;
        std::vector<double> ys;
        for (double v : y) ys.push_back((v - mean) / scale);
        const size_t d = Xs.empty() ? 0 : Xs[0].size();
        const double grid[] = {0.3, 0.45, 0.65, 0.9, 1.3, 2.0, 3.0};
        std::vector<double> l(d, 0.65);
        double best = -1e300, lml;
        if (fit_with(Xs, ys, l, 1e-3, &lml)) best = lml;
        for (int sweep = 0; sweep < 2; ++sweep)
            for (size_t k = 0; k < d; ++k) {
                double keep = l[k];
                for (double g : grid) {
                    l[k] = g;
                    if (fit_with(Xs, ys, l, 1e-3, &lml) && lml > best + 1e-9) {
                        best = lml;
                        keep = g;
                    }
                }
                l[k] = keep;
            }
        if (!fit_with(Xs, ys, l, 1e-3, &lml)) fit_with(Xs, ys, l, 1e-1, &lml);
    }

    // posterior mean and standard deviation in standardised units
    void predict(const std::vector<double> &x, double *mu, double *sd) const {
        std::vector<double> k(n);
        for (int i = 0; i < n; ++i) k[i] = matern52(x, X[i], ell);
        double m = 0.0;
        for (int i = 0; i < n; ++i) m += k[i] * alpha[i];
        solve_lower(L, n, k);
        double v = 1.0;
        for (double t : k) v -= t * t;
        *mu = m;
        *sd = std::sqrt(std::max(v, 1e-12));
    }
};

double norm_cdf(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }
double norm_pdf(double z) { return std::exp(-0.5 * z * z) / std::sqrt(2.0 * M_PI); }

}  // namespace

using CostFn = std::function<double(const bplg_plan &)>;

// Search over `plans`; writes the chosen index.  regs/smem (may be empty)
// feed the analytical method.
// Stopping window of the learned tuner: the search ends once this many
// evaluations in a row brought no new best.  Section IV-B uses 5 with
// GPTune's LCM surrogate; with this single-task GP a 5-evaluation window
// stopped early on the large tridiagonal spaces (1000-2000 plans), so the
// default is 8.  BPLG_BO_WINDOW (1..64) overrides it, e.g. 5 for the paper's.
static int bo_window() {
    static const int w = [] {
        const char *e = std::getenv("BPLG_BO_WINDOW");
        const int v = e ? std::atoi(e) : 0;
        return (v >= 1 && v <= 64) ? v : 8;
    }();
    return w;
}

// The learned-cost-model search (Section IV-B) in ask/tell form: next()
// names the plan to evaluate (-1 once the search has stopped) and tell()
// records its time.  tune_search runs it in a loop; the online tuner feeds
// it one real call at a time.
//   * Initial design: max(5, ceil(0.6 sqrt N)) (<= 24, <= budget) plans,
//     space-filling over the encoded knobs (the role of GPTune's
//     Latin-hypercube start): a seeded random first plan, then each next plan
//     the one farthest from those already chosen (largest minimum squared
//     distance; ties broken by a seeded random order).
//   * Then Gaussian-process expected improvement over the unevaluated plans,
//     log time as the target, invalid plans at 10x the worst time seen,
//     until the stopping window of evaluations without a new best, the
//     budget, or the space runs out.
struct BoSearch {
    int N = 0, budget = 0, n0 = 0, window = 0;
    std::vector<std::vector<double>> X;
    std::vector<int> perm;
    std::vector<double> dmin, ms;
    std::vector<char> seen;
    double best = INFINITY;
    int since = 0, evals = 0, n_invalid = 0;
    int init_next = -1;

    BoSearch(const std::vector<bplg_plan> &plans, int budget_, uint64_t seed) {
        N = static_cast<int>(plans.size());
        budget = budget_ > 0 ? budget_ : 40;
        SplitMix rng{seed ^ 0x5DEECE66Dull};
        n0 = static_cast<int>(std::ceil(0.6 * std::sqrt(static_cast<double>(N))));
        n0 = std::max(5, std::min(n0, 24));
        n0 = std::min(std::min(n0, N), budget);
        X = encode(plans);
        perm.resize(N);
        std::iota(perm.begin(), perm.end(), 0);
        for (int i = N - 1; i > 0; --i) {
            int j = static_cast<int>(rng.next() % uint64_t(i + 1));
            std::swap(perm[i], perm[j]);
        }
        dmin.assign(N, INFINITY);
        ms.assign(N, NAN);
        seen.assign(N, 0);
        window = bo_window();
        init_next = N > 0 ? perm[0] : -1;
    }

    int next() const {
        if (evals < n0) return init_next;
        if (!(evals < budget && evals < N && since < window)) return -1;
        std::vector<std::vector<double>> Xs;
        std::vector<double> ys;
        double ymax = -1e300;
        for (int i = 0; i < N; ++i)
            if (seen[i] && std::isfinite(ms[i])) ymax = std::max(ymax, std::log(ms[i]));
        if (ymax < -1e299) ymax = 0.0;
        for (int i = 0; i < N; ++i) {
            if (!seen[i]) continue;
            Xs.push_back(X[i]);
            ys.push_back(std::isfinite(ms[i]) ? std::log(ms[i]) : ymax + std::log(10.0));
        }
        GP gp;
        gp.fit(Xs, ys);
        const double ybest = std::isfinite(best) ? (std::log(best) - gp.mean) / gp.scale : 1e9;
        int pick = -1;
        double pick_ei = -1.0;
        for (int i = 0; i < N; ++i) {
            if (seen[i]) continue;
            double mu, sd;
            gp.predict(X[i], &mu, &sd);
            const double imp = ybest - mu - 0.01;
            const double z = imp / sd;
            const double ei = imp * norm_cdf(z) + sd * norm_pdf(z);
            if (ei > pick_ei) {
                pick_ei = ei;
                pick = i;
            }
        }
        return pick;
    }

    // record plan i's time (non-positive or non-finite: invalid)
    void tell(int i, double t) {
        if (i < 0 || i >= N || seen[i]) return;
        if (!(t > 0.0) || !std::isfinite(t)) {
            ++n_invalid;
            t = INFINITY;
        }
        ms[i] = t;
        seen[i] = 1;
        ++evals;
        if (evals <= n0) {
            if (t < best) best = t;
            int far = -1;
            double far_d = -1.0;
            for (int q = 0; q < N; ++q) {
                const int c = perm[q];
                if (seen[c]) continue;
                double d2 = 0.0;
                for (size_t f = 0; f < X[c].size(); ++f) {
                    const double u = X[c][f] - X[i][f];
                    d2 += u * u;
                }
                dmin[c] = std::min(dmin[c], d2);
                if (dmin[c] > far_d) {
                    far_d = dmin[c];
                    far = c;
                }
            }
            init_next = far;
            if (far < 0) n0 = evals;  // the space is exhausted
        } else if (t < best * (1.0 - 1e-3)) {
            best = t;
            since = 0;
        } else {
            ++since;
        }
    }

    int best_index() const {
        int b = -1;
        for (int i = 0; i < N; ++i)
            if (seen[i] && std::isfinite(ms[i]) && (b < 0 || ms[i] < ms[b])) b = i;
        return b;
    }
};

BoSearch *bo_create(const std::vector<bplg_plan> &plans, int budget, uint64_t seed) {
    return new BoSearch(plans, budget, seed);
}
int bo_next(const BoSearch *b) { return b->next(); }
void bo_tell(BoSearch *b, int i, double ms) { b->tell(i, ms); }
int bo_best(const BoSearch *b) { return b->best_index(); }
int bo_evaluations(const BoSearch *b) { return b->evals; }
void bo_destroy(BoSearch *b) { delete b; }

int tune_search(const std::vector<bplg_plan> &plans, const std::vector<int> &regs, const std::vector<int> &smem,
                const bplg_arch &arch, int method, int budget, uint64_t seed, const CostFn &cost, int *chosen,
                bplg_tune_report *rep, const std::vector<double> *model_times) {
    bplg_tune_report r;
    std::memset(&r, 0, sizeof(r));
    r.method = method;
    r.space_size = static_cast<int32_t>(plans.size());
    r.chosen_ms = NAN;
    r.best_seen_ms = NAN;
    *chosen = -1;
    if (plans.empty()) {
        if (rep) *rep = r;
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "empty search space");
    }
    const int N = static_cast<int>(plans.size());
    std::vector<double> ms(N, NAN);
    std::vector<char> seen(N, 0);
    auto evaluate = [&](int i) {
        double t = cost(plans[i]);
        ++r.evaluations;
        if (!(t > 0.0) || !std::isfinite(t)) {
            ++r.invalid;
            t = INFINITY;
        }
        ms[i] = t;
        seen[i] = 1;
        if (std::isfinite(t) && (!std::isfinite(r.best_seen_ms) || t < r.best_seen_ms)) r.best_seen_ms = t;
        return t;
    };
    auto best_index = [&]() {
        int b = -1;
        for (int i = 0; i < N; ++i)
            if (seen[i] && std::isfinite(ms[i]) && (b < 0 || ms[i] < ms[b])) b = i;
        return b;
    };

    if (method == BPLG_TUNE_ANALYTIC) {
        std::vector<bplg_candidate> c;
        for (int i = 0; i < N; ++i)
            c.push_back(to_candidate(plans[i], regs.empty() ? 32 : regs[i], smem.empty() ? 0 : smem[i]));
        const bool radix = plans[0].op == BPLG_OP_FFT || plans[0].op == BPLG_OP_FFT_TC;
        *chosen = guideline_select(arch, c.data(), N, radix);
        if (*chosen < 0) {
            if (rep) *rep = r;
            return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "no candidate can launch");
        }
    } else if (method == BPLG_TUNE_MODEL) {
        if (!model_times || model_times->size() != plans.size()) {
            if (rep) *rep = r;
            return set_error(BPLG_ERR_INVALID_ARG, "the cost model needs the plans' resources");
        }
        for (int i = 0; i < N; ++i)
            if (std::isfinite((*model_times)[i]) && (*chosen < 0 || (*model_times)[i] < (*model_times)[*chosen]))
                *chosen = i;
        if (*chosen < 0) {
            if (rep) *rep = r;
            return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "no candidate can launch");
        }
    } else if (method == BPLG_TUNE_EXHAUSTIVE) {
        for (int i = 0; i < N; ++i) evaluate(i);
        *chosen = best_index();
    } else if (method == BPLG_TUNE_LEARNED) {
        BoSearch bo(plans, budget, seed);
        for (int i = bo.next(); i >= 0; i = bo.next()) bo.tell(i, evaluate(i));
        *chosen = best_index();
    } else {
        if (rep) *rep = r;
        return set_error(BPLG_ERR_INVALID_ARG, "unknown tuning method");
    }
    if (*chosen < 0) {
        if (rep) *rep = r;
        return set_error(BPLG_ERR_INVALID_PLAN, "no candidate produced a valid time");
    }
    r.chosen_ms = seen[*chosen] ? ms[*chosen] : NAN;
    if (rep) *rep = r;
    return BPLG_OK;
}

// ---------------------------------------------------------- GPU timing
namespace {

__global__ void fill_kernel(int op, int dtype, int64_t n, int64_t total, void *p0, void *p1, void *p2,
                            void *p3) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint64_t z = static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull + 0x1234567ull;
        z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
        const float u = static_cast<float>((z >> 40) & 0xFFFFFF) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
        if (op == BPLG_OP_SCAN) {
            if (dtype == BPLG_I32)
                static_cast<int32_t *>(p0)[i] = static_cast<int32_t>(u * 1000.0f);
            else
                static_cast<float *>(p0)[i] = u;
        } else if (op == BPLG_OP_FFT || op == BPLG_OP_FFT_TC) {
            static_cast<float2 *>(p0)[i] = make_float2(u, -u * 0.5f);
        } else {
            static_cast<float *>(p0)[i] = (i % n) ? 0.5f * u : 0.f;
            static_cast<float *>(p1)[i] = 2.5f + 0.5f * u;
            static_cast<float *>(p2)[i] = ((i + 1) % n) ? -0.5f * u : 0.f;
            static_cast<float *>(p3)[i] = u;
        }
    }
}

struct TuneBuffers {
    void *in = nullptr, *out = nullptr, *b = nullptr, *c = nullptr, *d = nullptr;
    ~TuneBuffers() {
        for (void *p : {in, out, b, c, d})
            if (p) cudaFree(p);
    }
};

}  // namespace

int launch_plan(const bplg_plan &p, int dtype, int64_t n, int64_t batch, void *in, void *out, void *b,
                void *c, void *d, cudaStream_t s) {
    switch (p.op) {
        case BPLG_OP_SCAN: return scan_launch(p, dtype, in, out, n, batch, s);
        case BPLG_OP_FFT: return fft_launch(p, in, out, n, batch, -1, s);
        case BPLG_OP_FFT_TC: return fft_tc_launch(p, in, out, n, batch, -1, BPLG_TC_BF16, s);
        case BPLG_OP_TRIDIAG:
            return tridiag_launch(p, static_cast<const float *>(in), static_cast<const float *>(b),
                                  static_cast<const float *>(c), static_cast<const float *>(d),
                                  static_cast<float *>(out), n, batch, s);
        case BPLG_OP_TRIDIAG_WM:
            return tridiag_wm_launch(p, static_cast<const float *>(in), static_cast<const float *>(b),
                                     static_cast<const float *>(c), static_cast<const float *>(d),
                                     static_cast<float *>(out), n, batch, s);
        case BPLG_OP_TRIDIAG_REFINED:
            return tridiag_refined_launch(p, static_cast<const float *>(in), static_cast<const float *>(b),
                                          static_cast<const float *>(c), static_cast<const float *>(d),
                                          static_cast<double *>(out), n, batch, 10, 1e-14, nullptr, s);
        default: return set_error(BPLG_ERR_INVALID_ARG, "op cannot be timed");
    }
}

// Median time in ms of `reps` launches of plan p (after warm-up), each
// bracketed by CUDA events on `s`; +inf if a launch failed or the wall-clock
// limit passed.
double time_plan(const bplg_plan &p, int dtype, int64_t n, int64_t batch, int reps, void *in, void *out,
                 void *b, void *c, void *d, cudaStream_t s, double limit_s) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return INFINITY;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return INFINITY;
    }
    std::vector<double> t;
    const auto start = std::chrono::steady_clock::now();
    bool ok = true;
    for (int k = 0; k < reps + 2 && ok; ++k) {
        cudaEventRecord(e0, s);
        if (launch_plan(p, dtype, n, batch, in, out, b, c, d, s) != BPLG_OK) ok = false;
        cudaEventRecord(e1, s);
        while (ok) {
            cudaError_t q = cudaEventQuery(e1);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) {
                ok = false;
                break;
            }
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count() > limit_s) {
                ok = false;
                set_error(BPLG_ERR_TIMEOUT, "tuning candidate exceeded its wall-clock limit");
                break;
            }
        }
        float ms = 0.f;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            if (k >= 2) t.push_back(ms);
        } else {
            ok = false;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || t.empty()) return INFINITY;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// Library-owned buffers shaped like (op, dtype, n, batch), filled with
// well-conditioned values, plus a private stream: the timing arena of the
// tuners.
struct TimingArena {
    TuneBuffers tb;
    cudaStream_t s = nullptr;
    int op = 0, dtype = 0;
    int64_t n = 0, batch = 0;
    ~TimingArena() {
        if (s) cudaStreamDestroy(s);
    }
    int open(int op_, int dtype_, int64_t n_, int64_t batch_) {
        op = op_;
        dtype = dtype_;
        n = n_;
        batch = batch_;
        cudaError_t e;
        const int64_t total = n * batch;
        const bool cplx = op == BPLG_OP_FFT || op == BPLG_OP_FFT_TC;
        const size_t esz = cplx ? 8 : 4;
        const size_t osz = (cplx || op == BPLG_OP_TRIDIAG_REFINED) ? 8 : 4;
        if ((e = cudaMalloc(&tb.in, total * esz)) != cudaSuccess) return cuda_error(e, "timing buffers");
        if ((e = cudaMalloc(&tb.out, total * osz)) != cudaSuccess) return cuda_error(e, "timing buffers");
        if (op == BPLG_OP_TRIDIAG || op == BPLG_OP_TRIDIAG_REFINED || op == BPLG_OP_TRIDIAG_WM) {
            if ((e = cudaMalloc(&tb.b, total * 4)) != cudaSuccess) return cuda_error(e, "timing buffers");
            if ((e = cudaMalloc(&tb.c, total * 4)) != cudaSuccess) return cuda_error(e, "timing buffers");
            if ((e = cudaMalloc(&tb.d, total * 4)) != cudaSuccess) return cuda_error(e, "timing buffers");
        }
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_error(e, "timing stream");
        fill_kernel<<<1024, 256, 0, s>>>(op, dtype, n, total, tb.in, tb.b, tb.c, tb.d);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "timing fill");
        return BPLG_OK;
    }
    double time(const bplg_plan &p, int reps) {
        return time_plan(p, dtype, n, batch, reps, tb.in, tb.out, tb.b, tb.c, tb.d, s, 60.0);
    }
};

int time_plan_owned(const bplg_plan &p, int dtype, int64_t n, int64_t batch, int reps, double *ms) {
    TimingArena arena;
    int rc = arena.open(p.op, dtype, n, batch);
    if (rc != BPLG_OK) return rc;
    *ms = arena.time(p, reps);
    if (!std::isfinite(*ms)) return set_error(BPLG_ERR_CUDA, "timing failed");
    return BPLG_OK;
}

int tune_on_device(int op, int dtype, int64_t n, int64_t batch, int method, int budget, uint64_t seed,
                   bplg_plan *out, bplg_tune_report *rep) {
    bplg_arch a;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    int rc = arch_query(dev, &a);
    if (rc != BPLG_OK) return rc;
    std::vector<bplg_plan> plans;
    std::vector<int> regs, smem;
    rc = device_space(op, dtype, n, &plans, &regs, &smem);
    if (rc != BPLG_OK) return rc;
    if (plans.empty()) return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "no valid plan for this size");
    TimingArena arena;
    if (method == BPLG_TUNE_LEARNED || method == BPLG_TUNE_EXHAUSTIVE) {
        rc = arena.open(op, dtype, n, batch);
        if (rc != BPLG_OK) return rc;
    }
    std::vector<double> mt;
    if (method == BPLG_TUNE_MODEL) {
        rc = model_times_on_device(dev, plans, regs, smem, n, batch, &mt);
        if (rc != BPLG_OK) return rc;
    }
    const int reps = 25;
    CostFn cost = [&](const bplg_plan &p) { return arena.time(p, reps); };
    int chosen = -1;
    rc = tune_search(plans, regs, smem, a, method, budget, seed, cost, &chosen, rep, &mt);
    if (rc != BPLG_OK) return rc;
    *out = plans[chosen];
    cache_store(op, dtype, n, batch, *out);
    return BPLG_OK;
}

}  // namespace bplg
