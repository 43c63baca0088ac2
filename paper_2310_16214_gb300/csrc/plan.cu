// Plans: validity of a knob tuple for a problem size, canonical enumeration
// of the search space (Section IV-B, Table I; constraints of Section V
// restated for the GB300), shared-memory sizes, the per-process plan cache,
// and the per-device dynamic shared-memory opt-in.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <tuple>

#include "internal.h"

namespace bplg {

int fft_smem_bytes(int radix, int layout, int pad, int io, int64_t n, int spb);
int fft_tc_smem_bytes(int64_t n, int spb, int io);
bool fft_tc_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int prec, int dir, Launch *out);
int tridiag_smem_bytes(int pad, int64_t n, int spb, bool refined, int layout, int io, int log_m, int P);

namespace {
thread_local std::string t_last_error;
}

int set_error(int code, const std::string &msg) {
    t_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    t_last_error = m;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return BPLG_ERR_NO_DEVICE;
    return BPLG_ERR_CUDA;
}

void clear_error() { t_last_error.clear(); }

int check_grid(int64_t blocks, const char *what) {
    if (blocks >= 1 && blocks <= kMaxGridBlocks) return BPLG_OK;
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "%s: the batch needs %lld blocks, above the grid limit of 2^31 - 1; split the batch or use a plan "
                  "with more problems per block", what, static_cast<long long>(blocks));
    return set_error(BPLG_ERR_UNSUPPORTED_SIZE, buf);
}

int launch_error(cudaError_t e, const char *what, const void *func, int64_t grid, int threads, int smem) {
    char buf[512];
    cudaFuncAttributes fa;
    std::memset(&fa, 0, sizeof(fa));
    cudaError_t e2 = cudaFuncGetAttributes(&fa, func);
    std::snprintf(buf, sizeof(buf),
                  " [grid %lld, block %d, dynamic smem %d; kernel: regs %d, static smem %zu, local %zu, "
                  "max threads %d, max dynamic smem %d, attr query %s]",
                  static_cast<long long>(grid), threads, smem, fa.numRegs, fa.sharedSizeBytes, fa.localSizeBytes,
                  fa.maxThreadsPerBlock, fa.maxDynamicSharedSizeBytes, cudaGetErrorName(e2));
    int rc = cuda_error(e, what);
    t_last_error += buf;
    return rc;
}

const char *last_error_cstr() { return t_last_error.c_str(); }

static bool fail(std::string *why, const char *msg) {
    if (why) *why = msg;
    return false;
}

int max_log_for(int op) {
    switch (op) {
        case BPLG_OP_SCAN: return kScanMaxLog;
        case BPLG_OP_FFT: return kFftLargeMaxLog;
        case BPLG_OP_TRIDIAG: return kTridiagMaxLog;
        case BPLG_OP_TRIDIAG_REFINED: return kRefinedMaxLog;
        case BPLG_OP_TRIDIAG_WM: return kTridiagMaxLog;
        case BPLG_OP_FFT_TC: return kFftMaxLog;
        default: return -1;
    }
}

bool plan_structurally_valid(const bplg_plan &p, int dtype, int64_t n, std::string *why) {
    const int ml = max_log_for(p.op);
    if (ml < 0) return fail(why, "unknown op");
    if (!is_pow2(n) || n > (int64_t(1) << ml)) return fail(why, "n is not a supported power of two");
    if (p.n != 0 && p.n != n) return fail(why, "plan was made for another n");
    if (p.op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog)) return fft_large_plan_valid(p, n, why);
    if (p.n1_log != 0 || p.row_spb != 0 || p.reserved != 0)
        return fail(why, "n1_log, row_spb and reserved are 0 except for FFTs above 16384 points");
    if (!is_pow2(p.P) || p.P > 32 || p.P > n) return fail(why, "P must be a power of two <= min(32, n)");
    if (p.spb < 1) return fail(why, "spb must be >= 1");
    const int64_t tps = n / p.P;
    if (tps > 1024) return fail(why, "more than 1024 threads per problem");
    if (int64_t(p.spb) * tps != p.L) return fail(why, "L must equal spb * n / P");
    if (p.L < 32 || p.L > 1024 || (p.L & 31)) return fail(why, "L must be a multiple of 32 in [32, 1024]");
    switch (p.op) {
        case BPLG_OP_SCAN:
            if (dtype != BPLG_I32 && dtype != BPLG_F32) return fail(why, "scan dtype must be I32 or F32");
            if (p.pattern != BPLG_PATTERN_KS && p.pattern != BPLG_PATTERN_LF) return fail(why, "bad scan pattern");
            if (tps > 32 * 32) return fail(why, "scan: at most 32 warps per problem");
            return true;
        case BPLG_OP_FFT:
            if (p.radix != 2 && p.radix != 4 && p.radix != 8 && p.radix != 16) return fail(why, "radix must be 2, 4, 8 or 16");
            if (p.P != p.radix) return fail(why, "FFT: P must equal the radix");
            if (n < 2) return fail(why, "FFT: n >= 2");
            if (p.smem_layout < 0 || p.smem_layout > 1 || p.smem_pad < 0 || p.smem_pad > 1 || p.io < 0 || p.io > 2)
                return fail(why, "FFT: layout/pad/io out of range");
            if (p.smem_layout == 1 && p.io == 1) return fail(why, "FFT: staged io needs the interleaved layout");
            if (p.smem_layout == 1 && p.io == 2 && (p.radix != 16 || p.smem_pad != 1 || n < 1024 || n > 16384))
                return fail(why, "FFT: the split-exchange pipelined variant is radix 16, padded, 1024 <= n <= 16384");
            return true;
        case BPLG_OP_FFT_TC:
            if (p.io == 2) {
                if (p.radix != 16 || p.smem_pad != 1 || p.smem_layout != 0 ||
                    !((n == 4096 && p.P == 16 && p.spb == 2) || (n == 16384 && p.P == 32 && p.spb == 1)))
                    return fail(why, "tensor-core FFT, two 64-point GEMM passes (io 2): n = 4096 (P 16, spb 2) or "
                                     "16384 (P 32, spb 1), 512 threads, radix 16, padded interleaved");
                return true;
            }
            if (p.radix != 16 || p.P != 16) return fail(why, "tensor-core FFT: radix and P are 16");
            if (n < 512) return fail(why, "tensor-core FFT: n >= 512 (a warp per 32 butterflies)");
            if (p.smem_pad != 1 || p.smem_layout != 0 || p.io < 0 || p.io > 2)
                return fail(why, "tensor-core FFT: padded interleaved layout; io 0 (tcgen05), 1 (mma.sync) or 2 "
                                 "(two GEMM passes)");
            if (p.io == 0 && (n < 1024 || n > 16384 || p.L % 128 != 0))
                return fail(why, "tensor-core FFT with tcgen05: 1024 <= n <= 16384 and blocks of 128-thread tiles");
            return true;
        case BPLG_OP_TRIDIAG_WM:
            if (n < 2) return fail(why, "Wang-Mou: n >= 2");
            if (p.P < 2 || p.P > 16) return fail(why, "Wang-Mou: 2 <= P <= 16");
            if (p.radix != 2 && p.radix != 4 && p.radix != 8) return fail(why, "Wang-Mou: radix must be 2, 4 or 8");
            if (tps > 1 && p.radix > tps) return fail(why, "Wang-Mou: radix <= n / P");
            if (p.shuffle < 0 || p.shuffle > 1) return fail(why, "Wang-Mou: shuffle is 0 or 1");
            if (p.pattern != 0 || p.smem_layout != 0 || p.smem_pad != 0 || p.io != 0 || p.cr_switch != 0)
                return fail(why, "Wang-Mou: pattern, smem_layout, smem_pad, io and cr_switch are 0");
            return true;
        case BPLG_OP_TRIDIAG:
        case BPLG_OP_TRIDIAG_REFINED: {
            if (n < 2) return fail(why, "tridiag: n >= 2");
            if (p.P > 16) return fail(why, "tridiag: P <= 16");
            if (!is_pow2(p.cr_switch) || p.cr_switch > n || p.cr_switch > tps)
                return fail(why, "tridiag: cr_switch must be a power of two <= min(n, n/P)");
            if (p.shuffle < 0 || p.shuffle > 1 || p.smem_pad < 0 || p.smem_pad > 1)
                return fail(why, "tridiag: shuffle/pad out of range");
            if (p.shuffle && p.cr_switch > 32) return fail(why, "tridiag: shuffle PCR needs cr_switch <= 32");
            if (p.op == BPLG_OP_TRIDIAG_REFINED && tps < 32) return fail(why, "refined: at least 32 threads per system");
            if (p.smem_layout < 0 || p.smem_layout > (p.op == BPLG_OP_TRIDIAG_REFINED ? 7 : 2))
                return fail(why, "tridiag: smem_layout out of range (0 strided rows, 1 compacted levels, 2 register "
                                 "levels; refined: bit 0 float64 coefficients, bit 1 compacted levels, 4-6 register levels, "
                                 "7 Wang-Mou solves)");
            if (p.op == BPLG_OP_TRIDIAG && p.smem_layout == 2 && (p.P < 2 || (p.io == 1 && (p.P < 4 || n < 64))))
                return fail(why, "tridiag: register levels need P >= 2 (P >= 4 and n >= 64 when pipelined)");
            if (p.op == BPLG_OP_TRIDIAG && p.smem_layout == 1 && (p.smem_pad != 1 || p.io != 0))
                return fail(why, "tridiag: the compacted layout is always padded and per-block");
            if (p.op == BPLG_OP_TRIDIAG_REFINED && p.smem_layout < 4 && (p.smem_layout & 2) && p.smem_pad != 1)
                return fail(why, "refined: the compacted layout is always padded");
            if (p.op == BPLG_OP_TRIDIAG_REFINED && p.smem_layout >= 4 && (p.P < 2 || (p.smem_layout == 5 && p.P > 8)))
                return fail(why, "refined: register levels need P >= 2 (P <= 8 with float64 coefficients)");
            if (p.op == BPLG_OP_TRIDIAG_REFINED && p.smem_layout == 7 &&
                (p.shuffle != 1 || p.smem_pad != 0 || p.cr_switch != 32))
                return fail(why, "refined: the Wang-Mou layout takes shuffle 1, pad 0 and cr_switch 32 (unused)");
            if (p.io < 0 || p.io > (p.op == BPLG_OP_TRIDIAG ? 1 : 0))
                return fail(why, "tridiag: io out of range (0 per-block, 1 pipelined)");
            if (p.io == 1 && n < 4) return fail(why, "tridiag: the pipelined kernel needs n >= 4");
            return true;
        }
        default:
            return fail(why, "unknown op");
    }
}

int plan_smem_bytes(const bplg_plan &p, int dtype, int64_t n) {
    (void)dtype;
    if (p.op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog))
        return std::max(fft_large_smem_bytes(p, n, 0), fft_large_smem_bytes(p, n, 1));
    switch (p.op) {
        case BPLG_OP_SCAN: return 0;
        case BPLG_OP_FFT: return fft_smem_bytes(p.radix, p.smem_layout, p.smem_pad, p.io, n, p.spb);
        case BPLG_OP_FFT_TC: return fft_tc_smem_bytes(n, p.spb, p.io);
        case BPLG_OP_TRIDIAG:
            return tridiag_smem_bytes(p.smem_pad, n, p.spb, false, p.smem_layout, p.io, ilog2(p.cr_switch), p.P);
        case BPLG_OP_TRIDIAG_REFINED:
            return tridiag_smem_bytes(p.smem_pad, n, p.spb, true, p.smem_layout, 0, ilog2(p.cr_switch), p.P);
        case BPLG_OP_TRIDIAG_WM: return tridiag_wm_smem_bytes(p, n);
        default: return 0;
    }
}

void plan_finalize(bplg_plan *p, int dtype, int64_t n) {
    if (p->op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog)) {
        fft_large_finalize(p, n);
        return;
    }
    p->n = static_cast<int32_t>(n);
    const int64_t tps = p->P > 0 ? n / p->P : 0;
    p->L = static_cast<int32_t>(p->spb * tps);
    switch (p->op) {
        case BPLG_OP_SCAN:
            p->radix = 2;
            p->shuffle = 1;
            p->smem_layout = p->smem_pad = p->io = p->cr_switch = 0;
            p->S = tps > 32 ? p->L / 32 : 0;
            break;
        case BPLG_OP_FFT:
            p->radix = p->P;
            p->shuffle = 0;
            p->pattern = p->cr_switch = 0;
            p->S = plan_smem_bytes(*p, dtype, n) > 0 ? static_cast<int32_t>(p->spb * n) : 0;
            break;
        case BPLG_OP_FFT_TC:
            p->radix = 16;
            p->shuffle = p->pattern = p->cr_switch = p->smem_layout = 0;
            p->smem_pad = 1;
            if (p->io != 0 && p->io != 2) p->io = 1;
            p->S = static_cast<int32_t>(p->spb * n);
            break;
        case BPLG_OP_TRIDIAG:
        case BPLG_OP_TRIDIAG_REFINED:
            p->radix = 2;
            p->pattern = 0;
            if (p->op == BPLG_OP_TRIDIAG_REFINED) p->io = 0;
            p->S = static_cast<int32_t>(p->spb * n);
            break;
        case BPLG_OP_TRIDIAG_WM:
            p->pattern = p->smem_layout = p->smem_pad = p->io = p->cr_switch = 0;
            p->S = plan_smem_bytes(*p, dtype, n) > 0 ? p->L : 0;  // descriptor slots
            break;
        default:
            break;
    }
    p->n1_log = p->row_spb = p->reserved = 0;
}

std::vector<bplg_plan> enumerate_structural(int op, int dtype, int64_t n) {
    std::vector<bplg_plan> out;
    if (max_log_for(op) < 0 || !is_pow2(n) || n > (int64_t(1) << max_log_for(op))) return out;
    if (op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog)) return fft_large_enumerate(n);
    auto push = [&](bplg_plan p) {
        plan_finalize(&p, dtype, n);
        if (plan_structurally_valid(p, dtype, n, nullptr)) out.push_back(p);
    };
    for (int P = 1; P <= 32; P *= 2) {
        if (P > n) break;
        const int64_t tps = n / P;
        if (tps > 1024) continue;
        for (int L = 32; L <= 1024; L *= 2) {
            if (L < tps || L % tps) continue;
            const int spb = static_cast<int>(L / tps);
            bplg_plan p;
            std::memset(&p, 0, sizeof(p));
            p.op = op;
            p.P = P;
            p.spb = spb;
            if (op == BPLG_OP_SCAN) {
                for (int pat = 0; pat <= 1; ++pat) {
                    p.pattern = pat;
                    push(p);
                }
            } else if (op == BPLG_OP_TRIDIAG_WM) {
                for (int r = 8; r >= 2; r /= 2) {
                    for (int sh = 1; sh >= 0; --sh) {
                        p.radix = r;
                        p.shuffle = sh;
                        push(p);
                    }
                }
            } else if (op == BPLG_OP_FFT_TC) {
                p.radix = 16;
                if (P == 16) {
                    for (int io = 0; io <= 1; ++io) {
                        p.io = io;
                        push(p);
                    }
                }
                p.io = 2;  // the two-GEMM-pass kernel: valid for one (P, spb) per size
                push(p);
            } else if (op == BPLG_OP_FFT) {
                if (P < 2 || P > 16) continue;
                p.radix = P;
                const int io_order[3] = {2, tps >= 32 ? 0 : 1, tps >= 32 ? 1 : 0};
                for (int io_i = 0; io_i < 3; ++io_i) {
                    const int io = io_order[io_i];
                    for (int layout = 0; layout <= 1; ++layout) {
                        for (int pad = 1; pad >= 0; --pad) {
                            p.io = io;
                            p.smem_layout = layout;
                            p.smem_pad = pad;
                            push(p);
                        }
                    }
                }
            } else {
                const int64_t mmax = tps < n ? tps : n;
                const int layouts = op == BPLG_OP_TRIDIAG_REFINED ? 8 : 3;
                const int ios = op == BPLG_OP_TRIDIAG ? 2 : 1;
                for (int io = ios - 1; io >= 0; --io) {
                    for (int lay = layouts - 1; lay >= 0; --lay) {
                        for (int64_t m = mmax; m >= 1; m /= 2) {
                            for (int sh = 1; sh >= 0; --sh) {
                                for (int pad = 1; pad >= 0; --pad) {
                                    p.cr_switch = static_cast<int32_t>(m);
                                    p.shuffle = sh;
                                    p.smem_pad = pad;
                                    p.smem_layout = lay;
                                    p.io = io;
                                    push(p);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    return out;
}

// ------------------------------------------------------------ smem attribute
namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void *>, int> g_attr;  // (device, func) -> max dynamic smem set
}  // namespace

int ensure_smem_attr(const void *func, int smem) {
    if (smem <= 0) return BPLG_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_attr_mu);
    auto key = std::make_pair(dev, func);
    auto it = g_attr.find(key);
    if (it != g_attr.end() && it->second >= smem) return BPLG_OK;
    // the default limit (48 KB minus the kernel's static shared memory) is
    // kept when it suffices; otherwise opt in to the requested size
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes");
    if (fa.maxDynamicSharedSizeBytes < smem) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(max dynamic smem)");
    }
    g_attr[key] = smem;
    return BPLG_OK;
}

int persistent_grid(const void *func, int threads, int smem, int64_t items, int64_t *grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, int>, int64_t> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dev, func, threads, smem);
    auto it = cache.find(key);
    int64_t cap;
    if (it != cache.end()) {
        cap = it->second;
    } else {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, static_cast<size_t>(smem));
        if (e != cudaSuccess) return cuda_error(e, "occupancy query");
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
        cap = static_cast<int64_t>(per_sm > 0 ? per_sm : 1) * sms;
        cache[key] = cap;
    }
    *grid = items < cap ? items : cap;
    if (*grid < 1) *grid = 1;
    return BPLG_OK;
}

bool launch_info_for(const bplg_plan &p, int dtype, int64_t n, Launch *li) {
    switch (p.op) {
        case BPLG_OP_SCAN: return scan_launch_info(p, dtype, n, 1, li);
        case BPLG_OP_FFT:
            if (n > (int64_t(1) << kFftMaxLog)) return fft_large_launch_info(p, n, 1, -1, 0, li);
            return fft_launch_info(p, n, 1, -1, li);
        case BPLG_OP_TRIDIAG: return tridiag_launch_info(p, n, 1, false, li);
        case BPLG_OP_TRIDIAG_REFINED: return tridiag_launch_info(p, n, 1, true, li);
        case BPLG_OP_TRIDIAG_WM: return tridiag_wm_launch_info(p, n, 1, li);
        case BPLG_OP_FFT_TC: return fft_tc_launch_info(p, n, 1, BPLG_TC_BF16, -1, li);
        default: return false;
    }
}

static int check_launch_on_device(const Launch &li, std::string *why);

int check_plan_on_device(const bplg_plan &p, int dtype, int64_t n, std::string *why) {
    if (!plan_structurally_valid(p, dtype, n, why)) return BPLG_ERR_INVALID_PLAN;
    Launch li;
    if (!launch_info_for(p, dtype, n, &li)) {
        if (why) *why = "no kernel for this knob tuple";
        return BPLG_ERR_INVALID_PLAN;
    }
    if (p.op == BPLG_OP_FFT && n > (int64_t(1) << kFftMaxLog)) {  // the row kernel too
        Launch l2;
        if (!fft_large_launch_info(p, n, 1, -1, 1, &l2)) {
            if (why) *why = "no row kernel for this knob tuple";
            return BPLG_ERR_INVALID_PLAN;
        }
        const int rc = check_launch_on_device(l2, why);
        if (rc != BPLG_OK) return rc;
    }
    return check_launch_on_device(li, why);
}

static int check_launch_on_device(const Launch &li, std::string *why) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, li.func);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes");
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    if (li.threads > fa.maxThreadsPerBlock) {
        if (why) *why = "block larger than the kernel's thread limit";
        return BPLG_ERR_INVALID_PLAN;
    }
    if (static_cast<int64_t>(li.smem) + static_cast<int64_t>(fa.sharedSizeBytes) > optin) {
        if (why) *why = "shared memory above the per-block limit";
        return BPLG_ERR_INVALID_PLAN;
    }
    return BPLG_OK;
}

// ------------------------------------------------------------- plan cache
namespace {
std::mutex g_cache_mu;
std::map<std::tuple<int, int, int64_t, int>, bplg_plan> g_cache;
bool g_cache_loaded = false;

int batch_class(int64_t batch) { return ilog2(batch < 1 ? 1 : batch); }

const char *cache_file() {
    const char *f = std::getenv("BPLG_PLAN_CACHE");
    return (f && *f) ? f : nullptr;
}

void load_cache_locked() {
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char *f = cache_file();
    if (!f) return;
    std::ifstream in(f);
    std::string line;
    while (std::getline(in, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream ss(line);
        int op, dtype, bc;
        int64_t n;
        bplg_plan p;
        std::memset(&p, 0, sizeof(p));
        if (!(ss >> op >> dtype >> n >> bc >> p.op >> p.n >> p.P >> p.L >> p.spb >> p.S >> p.radix >> p.shuffle >>
              p.pattern >> p.smem_layout >> p.smem_pad >> p.io >> p.cr_switch))
            continue;
        int n1 = 0, rs = 0;
        if (ss >> n1 >> rs) {
            p.n1_log = n1;
            p.row_spb = rs;
        }
        if (plan_structurally_valid(p, dtype, n, nullptr)) g_cache[std::make_tuple(op, dtype, n, bc)] = p;
    }
}

void save_cache_locked() {
    const char *f = cache_file();
    if (!f) return;
    std::ofstream out(f, std::ios::trunc);
    out << "# op dtype n batch_log2 | op n P L spb S radix shuffle pattern layout pad io cr_switch n1_log row_spb\n";
    for (const auto &kv : g_cache) {
        const bplg_plan &p = kv.second;
        out << std::get<0>(kv.first) << ' ' << std::get<1>(kv.first) << ' ' << std::get<2>(kv.first) << ' '
            << std::get<3>(kv.first) << ' ' << p.op << ' ' << p.n << ' ' << p.P << ' ' << p.L << ' ' << p.spb << ' '
            << p.S << ' ' << p.radix << ' ' << p.shuffle << ' ' << p.pattern << ' ' << p.smem_layout << ' '
            << p.smem_pad << ' ' << p.io << ' ' << p.cr_switch << ' ' << p.n1_log << ' ' << p.row_spb << '\n';
    }
}
}  // namespace

bool cache_lookup(int op, int dtype, int64_t n, int64_t batch, bplg_plan *out) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_cache_locked();
    auto it = g_cache.find(std::make_tuple(op, dtype, n, batch_class(batch)));
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

void cache_store(int op, int dtype, int64_t n, int64_t batch, const bplg_plan &p) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_cache_locked();
    g_cache[std::make_tuple(op, dtype, n, batch_class(batch))] = p;
    save_cache_locked();
}

}  // namespace bplg
