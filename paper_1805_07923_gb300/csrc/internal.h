// Internal declarations of the MLSDC-SH library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "mlsdc_sh.h"
#include "node_update.cuh"
#include "vblock.cuh"

namespace mlsdc {

// thread-local text of the last CUDA error
void set_error(const char* where, cudaError_t e);
void set_error_text(const std::string& s);

// Record why an argument was refused; returns MLSDC_ERR_INVALID.
mlsdc_status invalid_arg(const std::string& why);

// The kernels read complex arrays as 16-byte double2 words, so a device
// pointer at an odd double offset (a flat float64 view sliced at [1:], say)
// would fault on the GPU.  Entry points refuse such pointers before any
// launch: MLSDC_ERR_INVALID with the offending argument named.  Null
// pointers pass here (each entry point checks those itself).
mlsdc_status check_aligned16(const char* where, std::initializer_list<std::pair<const char*, const void*>> ptrs);
#define MLSDC_ALIGNED(where, ...)                                          \
    do {                                                                   \
        mlsdc_status s_ = ::mlsdc::check_aligned16(where, {__VA_ARGS__});  \
        if (s_ != MLSDC_OK) return s_;                                     \
    } while (0)

#define MLSDC_CUDA(call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            ::mlsdc::set_error(#call, e_);                \
            return MLSDC_ERR_CUDA;                        \
        }                                                 \
    } while (0)

#define MLSDC_LAUNCHED(name)                              \
    do {                                                  \
        cudaError_t e_ = cudaGetLastError();              \
        if (e_ != cudaSuccess) {                          \
            ::mlsdc::set_error(name, e_);                 \
            return MLSDC_ERR_CUDA;                        \
        }                                                 \
    } while (0)

inline int nc_of(int R) { return (R + 1) * (R + 2) / 2; }

// Programmatic dependent launch.  The step's kernels are launched with
// programmatic stream serialisation, so a kernel's CTAs may start while its
// predecessor in the stream is still running; every kernel therefore calls
// pdl_wait() before its first global access that depends on, or could race
// with, an earlier kernel (reads of its inputs, any write), and only
// constant tables are touched before it.  pdl_wait() returns at once for a
// kernel launched without the attribute.  pdl_launch() lets the successor
// start its own prologue; it carries no memory guarantee (the successor's
// pdl_wait() waits for this grid to complete and its writes to be visible).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Whether launches use programmatic stream serialisation (off unless the
// environment sets MLSDC_PDL=1).
bool pdl_enabled();

// Programmatic serialisation for the launches made on this thread while a
// PdlScope(true) is alive, whatever pdl_enabled() says: for a kernel whose
// set-up before pdl_wait() (tensor memory, barriers, the first table tiles)
// is worth running beside its predecessor's tail.  Used for the
// tensor-core analysis after the FFT kernel; measured on the split-BF16
// step (150-step runs, two boxes): 1070 -> 1076 and 1081 steps/s.  The same
// for the synthesis, the FFT, the node updates or the transfers made the
// step slower (FFT 994, node updates 1045, transfers 1068): their
// successors' CTAs then sit on SMs the predecessor still needs.
bool& pdl_scope_flag();
struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(pdl_scope_flag()) { pdl_scope_flag() = prev || on; }
    ~PdlScope() { pdl_scope_flag() = prev; }
};

// One shared-memory carveout for every kernel launched through launch_k:
// two thirds of the SM's configurable L1/shared memory as shared memory.
// An SM switches its L1/shared split only when idle, so a sequence of
// dependent kernels that ask for different splits pays a drain at every
// change; measured on the split-BF16 step (3 x 150 steps, one box):
// per-kernel default 986 steps/s, 0 % 750, 50 % 922, 67 % 1027, 75 % 1019,
// 100 % 977.  A kernel whose shared memory does not fit the preference
// still gets the split it needs.
constexpr int kCarveoutPct = 67;
void set_carveout_once(const void* kernel);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
    if (Recorder* r = active_recorder()) {  // a kernel the persistent kernel has no body for
        r->refused = true;
        return cudaErrorNotSupported;
    }
    set_carveout_once((const void*)kernel);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = (pdl_enabled() || pdl_scope_flag()) ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// launch_k for a kernel whose body the persistent ensemble kernel can run:
// with a recorder installed on this thread the launch is recorded (body,
// grid, the shared memory the body needs: `smem` plus `static_smem` that the
// kernel itself declares, tensor-memory columns per block, packed
// arguments) instead of issued.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_b(Body body, int tmem_cols, size_t static_smem, void (*kernel)(KArgs...), dim3 grid,
                            dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    if (Recorder* r = active_recorder()) {
        record_launch(r, body, tmem_cols, smem + static_smem, kernel, grid, block, std::forward<Args>(args)...);
        return cudaSuccess;
    }
    return launch_k(kernel, grid, block, smem, st, std::forward<Args>(args)...);
}

#define MLSDC_LAUNCH(name, call)                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            ::mlsdc::set_error(name, e_);                 \
            return MLSDC_ERR_CUDA;                        \
        }                                                 \
    } while (0)

// Stage timing for the measurement entry points: `enqueue(stream)` issued
// `reps` times is captured into one CUDA graph, replayed once to warm up and
// once timed with CUDA events on `st`; *ms = milliseconds per enqueue.
// Inside a graph the per-launch cost is the device's (about 1.1 us per
// dependent kernel here), not the host's launch rate, as in the step graphs.
template <class Enqueue>
inline mlsdc_status time_in_graph(cudaStream_t st, int reps, float* ms, Enqueue enqueue) {
    cudaStream_t cap = nullptr;
    MLSDC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    mlsdc_status s = MLSDC_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    for (int r = 0; r < reps && s == MLSDC_OK && e == cudaSuccess; ++r) s = enqueue(cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaGraphInstantiate(&ge, g, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventCreate(&e0);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess && s == MLSDC_OK) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (s != MLSDC_OK) return s;
    if (e != cudaSuccess) {
        set_error("time_in_graph", e);
        return MLSDC_ERR_CUDA;
    }
    *ms = t / reps;
    return MLSDC_OK;
}

// Raise (never lower) a kernel's dynamic shared-memory limit.  The attribute
// belongs to the kernel, not to a plan, so a plan needing less must not undo
// the setting another live plan relies on.
mlsdc_status raise_smem_limit(const void* fn, size_t bytes);
__host__ __device__ inline int moff(int R, int m) { return m * (R + 1) - m * (m - 1) / 2; }

// Work item of a Legendre kernel: zonal wavenumber m and the first
// latitude (synthesis) or the first degree offset n - m (analysis).
struct Chunk {
    int m;
    int start;
};

// 2-D tensor maps over the float32 synthesis tables P32 and H32 ([nc][J2]
// floats, boxes of min(32, J2) latitudes x 32 rows, no swizzle): the float32
// synthesis can stream each work item's table rows into shared memory by TMA.
struct SynMaps {
    CUtensorMap P, H;
};
constexpr int kSynBoxRows = 32;

// Encode a 2-D float32 tensor map over a row-major [rows][cols] array with a
// box of box_cols x box_rows and no swizzle (false if the driver refuses).
bool make_rows_map_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                       uint32_t box_rows);

// Mixed-precision tables and scratch of a plan (float32 path).
struct MPTables {
    float* P32 = nullptr;        // [nc][J2] float32 copy of P
    float* H32 = nullptr;        // [nc][J2]
    float2* tw32 = nullptr;      // [I/2] float32 twiddles
    float2* stab32 = nullptr;    // [I/2] float32 stage-twiddle table of the radix-4 FFTs (I/2 - 1 used)
    float2* four_in = nullptr;   // [4][J][R+1]
    float2* four_out = nullptr;  // [5][R+1][J] (latitude-contiguous)
    float* lat32 = nullptr;      // [J][4] float32 copy of the plan's d_lat
    float* invnn32 = nullptr;    // [R+1] float32 copy of d_invnn
    SynMaps syn_maps;            // TMA maps of P32 / H32 for the float32 synthesis
    bool syn_tma = false;        // false: the synthesis reads the tables with plain loads (J2 % 4 != 0)
    int syn_tma_mode = 0;        // 0: by size (synth_uses_tma), 1: TMA whenever syn_tma, 2: plain loads
    int* d_err = nullptr;        // error word of the float32 synthesis's bounded TMA waits
    // tensor-core state (legendre_tc.cu): operand tables, tensor maps, error flag
    void* tc = nullptr;
    int64_t tc_bytes = 0;
    // tensor-core plans: which kernel each Legendre stage runs (kStageAuto:
    // by truncation and batch size, see stage_uses_tc; kStageTc: tcgen05;
    // kStageSimt: the float32 CUDA-core kernel)
    int synth_mode = 0, anal_mode = 0;
};

}  // namespace mlsdc

struct sh_plan_s {
    int R, I, J, J2, nc, logI, precision;
    int max_members = 1;              // ensemble members one F_E launch may carry
    std::vector<double> mu, w;        // host copies, north to south, length J
    double* d_mu = nullptr;           // [J]
    double* d_w = nullptr;            // [J]
    double* d_P = nullptr;            // [nc][J2], northern latitudes
    double* d_H = nullptr;            // [nc][J2]
    double2* d_tw = nullptr;          // [I/2] exp(-2 pi i k / I)
    double2* d_stab = nullptr;        // [I/2] stage-twiddle table of the radix-4 FFTs (I/2 - 1 used)
    int* d_ndeg = nullptr;            // [nc] total degree n of each coefficient
    double* d_cor = nullptr;          // [nc][4] Coriolis factors alpha, beta, gamma, 0 (coriolis_add)
    // Per-latitude and per-degree constants, computed on the host in float64
    // so no kernel divides in float64 (about 1/64 of the float32 rate here):
    double* d_lat = nullptr;          // [J][4] mu, 1/(1-mu^2), w/((1-mu^2) I), w/I
    double* d_invnn = nullptr;        // [R+1] 1/(n(n+1)), 0 for n = 0
    mlsdc::Chunk* d_synth = nullptr;  // synthesis work items, largest first
    mlsdc::Chunk* d_anal = nullptr;   // analysis work items, largest first
    int n_synth = 0, n_anal = 0;
    double2* d_four_in = nullptr;     // [max(16, 4 members)][J][R+1] Fourier coefficients (synthesis out)
    double2* d_four_out = nullptr;    // [max(16, 5 members)][J][R+1] Fourier coefficients (analysis in)
    mlsdc::MPTables mp;
    int64_t bytes = 0;
};

namespace mlsdc {
// chunk sizes of the float64 Legendre kernels
constexpr int kSynthLat = 32;   // latitudes per synthesis work item (one warp)
constexpr int kAnalRows = 32;   // degrees per analysis work item (one warp)
constexpr int kMaxFields = 16;

// Members of one F_E launch: `members` states `state_ms` complex values
// apart, results `fe_ms` apart.
struct RhsBatch {
    int members = 1;
    size_t state_ms = 0, fe_ms = 0;
};

// float64 kernels (transform_f64.cu)
// stage < 0: the whole F_E evaluation; 0, 1, 2: only that stage's kernel
mlsdc_status rhs_explicit_f64(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                              cudaStream_t st, int64_t* launches, int stage = -1, RhsBatch b = RhsBatch());
mlsdc_status f64_prepare(sh_plan_t p);
// float32 / tensor-core path (transform_mp.cu)
mlsdc_status mp_init(sh_plan_t p);
void mp_free(sh_plan_t p);
mlsdc_status rhs_explicit_mp(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                             cudaStream_t st, int64_t* launches, int stage = -1, RhsBatch b = RhsBatch());
mlsdc_status create_plan(int R, int nlon, int nlat, int precision, int max_members, sh_plan_t* out);
// whether a Legendre stage (0 synthesis, 2 analysis) of a tensor-core plan
// runs the tcgen05 kernel for a launch of `members` states (transform_mp.cu)
bool stage_uses_tc(const sh_plan_s* p, int stage, int members);
// pointwise float64 kernels (sdc.cu)
mlsdc_status implicit_rhs_launch(sh_plan_t p, const swe_params* prm, const double* state, double* FI,
                                 cudaStream_t st);
}  // namespace mlsdc
