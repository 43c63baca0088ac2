// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bplg.h"

namespace bplg {

// thread-local last-error message; returns `code` for convenient tail calls
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);
// cuda_error plus the launch geometry and the kernel's attributes
int launch_error(cudaError_t e, const char *what, const void *func, int64_t grid, int threads, int smem);
void clear_error();

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << (l + 1)) <= v) ++l;
    return l;
}
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Kernel function pointer plus the launch geometry derived from a plan.
struct Launch {
    const void *func = nullptr;  // __global__ function (for attributes)
    int threads = 0;             // threads per block
    int smem = 0;                // dynamic shared memory bytes
    int64_t blocks = 0;          // grid size
};

// Largest sizes each family supports.
constexpr int kScanMaxLog = 15;
constexpr int kFftMaxLog = 14;       // one block per signal
constexpr int kFftLargeMaxLog = 24;  // two-kernel transforms beyond that
constexpr int kTridiagMaxLog = 13;
constexpr int kRefinedMaxLog = 12;

// Largest grid (x dimension) of one launch: 2^31 - 1 blocks.
constexpr int64_t kMaxGridBlocks = 2147483647;
// BPLG_OK, or BPLG_ERR_UNSUPPORTED_SIZE (with a message naming `what`) when
// a launch would need more than kMaxGridBlocks blocks (batch too large for
// the plan's problems per block)
int check_grid(int64_t blocks, const char *what);

// ---- per-op kernel tables (each returns false if the plan has no kernel)
bool scan_launch_info(const bplg_plan &p, int dtype, int64_t n, int64_t batch, Launch *out);
int scan_launch(const bplg_plan &p, int dtype, const void *in, void *out, int64_t n, int64_t batch,
                cudaStream_t s);

bool fft_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int dir, Launch *out);
int fft_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir,
               cudaStream_t s);

int fft_tc_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir, int prec,
                  cudaStream_t s);

// two-kernel FFT for n > 2^kFftMaxLog (fft_large.cu); pass 0 = columns, 1 = rows
bool fft_large_plan_valid(const bplg_plan &p, int64_t n, std::string *why);
void fft_large_finalize(bplg_plan *p, int64_t n);
std::vector<bplg_plan> fft_large_enumerate(int64_t n);
int fft_large_smem_bytes(const bplg_plan &p, int64_t n, int pass);
bool fft_large_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int dir, int pass, Launch *out);
int fft_large_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir,
                     cudaStream_t s);

bool tridiag_launch_info(const bplg_plan &p, int64_t n, int64_t batch, bool refined, Launch *out);
int tridiag_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                   const float *d, float *x, int64_t n, int64_t batch, cudaStream_t s);
// Wang-Mou divide-and-conquer solver (tridiag_wm.cu)
int tridiag_wm_smem_bytes(const bplg_plan &p, int64_t n);
bool tridiag_wm_launch_info(const bplg_plan &p, int64_t n, int64_t batch, Launch *out);
int tridiag_wm_launch(const bplg_plan &p, const float *a, const float *b, const float *c, const float *d, float *x,
                      int64_t n, int64_t batch, cudaStream_t s);
int tridiag_refined_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                           const float *d, double *x, int64_t n, int64_t batch, int max_iter,
                           double tol, int32_t *iters, cudaStream_t s);

// ---- plans
// structural validity (sizes, knob ranges, geometry); no device query
bool plan_structurally_valid(const bplg_plan &p, int dtype, int64_t n, std::string *why);
// structural validity + device limits (threads, shared memory, registers)
int check_plan_on_device(const bplg_plan &p, int dtype, int64_t n, std::string *why);
// canonical enumeration of the structurally valid plans
std::vector<bplg_plan> enumerate_structural(int op, int dtype, int64_t n);
// shared memory (dynamic) a plan needs, in bytes
int plan_smem_bytes(const bplg_plan &p, int dtype, int64_t n);
// make S consistent with the other knobs
void plan_finalize(bplg_plan *p, int dtype, int64_t n);

// raise the dynamic shared-memory limit of `func` once per device
int ensure_smem_attr(const void *func, int smem);
// grid of a persistent kernel: min(work items, SMs x resident blocks per SM)
int persistent_grid(const void *func, int threads, int smem, int64_t items, int64_t *grid);

// ---- learned search in ask/tell form (tune.cu)
struct BoSearch;
BoSearch *bo_create(const std::vector<bplg_plan> &plans, int budget, uint64_t seed);
int bo_next(const BoSearch *b);  // plan index to evaluate next, -1 once stopped
void bo_tell(BoSearch *b, int i, double ms);
int bo_best(const BoSearch *b);  // best valid plan seen, -1 if none
int bo_evaluations(const BoSearch *b);
void bo_destroy(BoSearch *b);

// ---- GB300 analytical cost model (tune.cu)
struct DevModel {
    bplg_arch arch;
    double clk;  // sustained SM clock, Hz
    double bw;   // sustained HBM bandwidth, bytes/s
};
DevModel dev_model_from_arch(const bplg_arch &a, double peak_clock_hz, double nominal_bw);
int dev_model_query(int dev, DevModel *out);
double model_plan_time(const bplg_plan &p, int64_t n, int64_t batch, int regs, int smem, int regs2, int smem2,
                       const DevModel &dm);

// ---- plan cache (per process) and defaults
bool cache_lookup(int op, int dtype, int64_t n, int64_t batch, bplg_plan *out);
void cache_store(int op, int dtype, int64_t n, int64_t batch, const bplg_plan &p);
int analytic_plan(int op, int dtype, int64_t n, bplg_plan *out);

// library-owned device scratch per (device, stream, tag) (fft_large.cu)
constexpr int kScratchLargeFft = 0;
constexpr int kScratchBluestein = 1;
int stream_scratch(int tag, size_t bytes, cudaStream_t s, void **out);

// FFT of a length that is not a power of two (fft_bluestein.cu): Bluestein's
// chirp identity over power-of-two FFTs of size M >= 2n - 1 (plan: one for M,
// or NULL)
// mixed-radix Stockham FFT (radices 2 .. 16 whose factors are 2, 3, 5) for
// n = 2^a 3^b 5^c, not a power of two, n <= kMixedMaxN: one compile-time
// kernel per length (fft_mixed.cuh)
constexpr int64_t kMixedMaxN = 12288;
bool fft_mixed_supported(int64_t n);
int fft_mixed_launch(const void *in, void *out, int64_t n, int64_t batch, int dir, cudaStream_t s);
constexpr int kBluesteinMaxLog = 23;
int fft_bluestein_launch(const bplg_plan *plan_m, const void *in, void *out, int64_t n, int64_t batch, int dir,
                         cudaStream_t s);

// twiddle table of the current device (float2 W_M^k at [M + k], M = 2..2^14)
int twiddles_for_current_device(const void **tw);

}  // namespace bplg
