// Tensor-core Legendre contractions for MLSDC_TF32 and MLSDC_BF16X3 on
// sm_103a: tcgen05.mma with accumulators in tensor memory, the Legendre
// table tiles brought into shared memory by TMA (cp.async.bulk.tensor,
// 128-byte swizzle), a two-stage pipeline over K, and ensemble members
// batched along N.
//
// Synthesis (Eq. spectral_to_physical_space, the Legendre sum per m), one CTA
// per (zonal wavenumber m, chunk of members):
//   D[lat, 16 b + c] = sum_k A[lat, k] B[16 b + c, k],  A = P^m_{m+k}(mu_lat) or H^m_{m+k},
//   M = 128 northern latitudes (zero padded), K = degrees n - m in blocks of
//   128 bytes, and per member b 16 columns: the real and imaginary parts of
//   the coefficients (zeta, Phi', chi, psi for P; psi, chi for H) in two
//   column groups, one holding the even-(n-m) coefficients and one the odd
//   ones, so that north = even + odd and south = even - odd (H: odd - even).
// Analysis (Eq. legendre_transform), one CTA per (m, 128 degrees, member chunk):
//   D[k, 16 b + c] = sum_lat A[k, lat] B[16 b + c, lat],  A = P or H rows,
//   K = latitudes, B = each member's weighted Fourier coefficients of A..E
//   combined north + south (even) and north - south (odd); each row picks
//   its parity's columns.  The Coriolis part is added exactly in float64.
// TF32: operands rounded to tf32 (round to nearest); BF16X3: x = hi + lo in
// bf16 and D += A_hi B_hi + A_hi B_lo + A_lo B_hi.  Accumulation is float32
// in tensor memory; the final combination of F_E is float64.  With N = 16 x
// members per CTA (up to 256) a batch of members turns the skinny per-member
// contraction into a dense one.
//
// Every wait is bounded; on timeout the kernel records an error code in
// device memory (read by sh_plan_device_error), releases its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "complex.cuh"
#include "internal.h"
#include "legendre_tc.cuh"
#include "rhs_kernels.cuh"

namespace mlsdc {
namespace {

using namespace tc;

// each kernel's recorded arguments are its body's (persistent.cu)
MLSDC_SAME_PACK(k_tc_synth<MODE_BF16X3>, b_tc_synth<MODE_BF16X3>);
MLSDC_SAME_PACK(k_tc_anal<MODE_BF16X3>, b_tc_anal<MODE_BF16X3>);
MLSDC_SAME_PACK(k_tc_anal_ws<MODE_BF16X3>, b_tc_anal_ws<MODE_BF16X3>);

struct TcState {
    int mode = 0;
    int KS = 0;   // padded synthesis K (multiple of 64)
    int J2p = 0;  // padded analysis K (multiple of 64)
    void* syn[4] = {nullptr, nullptr, nullptr, nullptr};
    void* ana[4] = {nullptr, nullptr, nullptr, nullptr};
    Maps map_syn, map_ana;
    int* d_err = nullptr;
    int2* d_tiles = nullptr;
    int n_tiles = 0;
    // launch configuration per Legendre stage ([0] synthesis, [1] analysis;
    // autotuned): members per CTA, K pipeline depth, and for the analysis
    // whether batched launches run the warp-specialised kernel
    struct Cfg {
        int chunk = 1, stages = 0, ws = 0;
    } cfg[2];
};

// ---------------------------------------------------------- table builders
// Synthesis tables, K-major in n: row (m, lat) of length KS.
template <int MODE>
__global__ void k_build_syn(const double* __restrict__ T, int R, int J2, int KS, void* hi, void* lo) {
    const size_t total = (size_t)(R + 1) * kTileRows * KS;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % KS);
        const int row = (int)(i / KS);
        const int m = row / kTileRows, j = row % kTileRows;
        const int nm = R + 1 - m;
        float v = 0.f;
        if (j < J2 && k < nm) v = (float)T[(size_t)(m * (R + 1) - m * (m - 1) / 2 + k) * J2 + j];
        if (MODE == MODE_TF32) {
            reinterpret_cast<uint32_t*>(hi)[i] = to_tf32(v);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16*>(hi)[i] = h;
            reinterpret_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}
// Analysis tables, K-major in latitude: row (m, n) of length J2p.
template <int MODE>
__global__ void k_build_ana(const double* __restrict__ T, int nc, int J2, int J2p, void* hi, void* lo) {
    const size_t total = (size_t)nc * J2p;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % J2p);
        const size_t row = i / J2p;
        const float v = j < J2 ? (float)T[row * J2 + j] : 0.f;
        if (MODE == MODE_TF32) {
            reinterpret_cast<uint32_t*>(hi)[i] = to_tf32(v);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16*>(hi)[i] = h;
            reinterpret_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D tensor map over a row-major [rows][cols] table, box 128 B x 128 rows, 128-B swizzle.
bool make_map(CUtensorMap* map, void* base, int mode, uint64_t cols, uint64_t rows) {
    auto enc = get_encode();
    if (!enc) return false;
    const int esz = mode == MODE_TF32 ? 4 : 2;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)kTileRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, mode == MODE_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

TcState* st_of(sh_plan_t p) { return reinterpret_cast<TcState*>(p->mp.tc); }

constexpr size_t kSmemBudget = 227 * 1024;

// Pipeline depth for a member chunk: two stages when they fit, else one.
int stages_for(int mode, int chunk) {
    if (cta_smem_bytes(mode, chunk, 2) <= kSmemBudget) return 2;
    if (cta_smem_bytes(mode, chunk, 1) <= kSmemBudget) return 1;
    return 0;
}

template <int MODE>
mlsdc_status build_tables(sh_plan_t p, TcState* s) {
    const int esz = MODE == MODE_TF32 ? 4 : 2;
    const size_t nsyn = (size_t)(p->R + 1) * kTileRows * s->KS;
    const size_t nana = (size_t)p->nc * s->J2p;
    const int nparts = MODE == MODE_TF32 ? 1 : 2;
    for (int t = 0; t < 2; ++t)
        for (int q = 0; q < nparts; ++q) {
            MLSDC_CUDA(cudaMalloc(&s->syn[t * nparts + q], nsyn * esz));
            MLSDC_CUDA(cudaMalloc(&s->ana[t * nparts + q], nana * esz));
            p->mp.tc_bytes += (int64_t)(nsyn + nana) * esz;
        }
    for (int t = 0; t < 2; ++t) {
        const double* src = t == 0 ? p->d_P : p->d_H;
        void* sh = s->syn[t * nparts];
        void* sl = nparts == 2 ? s->syn[t * nparts + 1] : nullptr;
        void* ah = s->ana[t * nparts];
        void* al = nparts == 2 ? s->ana[t * nparts + 1] : nullptr;
        k_build_syn<MODE><<<1024, 256>>>(src, p->R, p->J2, s->KS, sh, sl);
        k_build_ana<MODE><<<1024, 256>>>(src, p->nc, p->J2, s->J2p, ah, al);
        MLSDC_LAUNCHED("k_build_tables");
    }
    MLSDC_CUDA(cudaDeviceSynchronize());
    for (int q = 0; q < 2 * nparts; ++q) {
        if (!make_map(&s->map_syn.m[q], s->syn[q], MODE, s->KS, (uint64_t)(p->R + 1) * kTileRows) ||
            !make_map(&s->map_ana.m[q], s->ana[q], MODE, s->J2p, (uint64_t)p->nc)) {
            set_error_text("cuTensorMapEncodeTiled failed or is unavailable");
            return MLSDC_ERR_CUDA;
        }
    }
    return MLSDC_OK;
}

template <int MODE>
mlsdc_status launch_synth(sh_plan_t p, TcState* s, const TcArgs& g, cudaStream_t st) {
    const int nchunks = (g.members + g.chunk - 1) / g.chunk;
    const size_t smem = cta_smem_bytes(MODE, g.chunk, g.stages);
    mlsdc_status rs = raise_smem_limit((const void*)k_tc_synth<MODE>, smem);
    if (rs != MLSDC_OK) return rs;
    MLSDC_LAUNCH("k_tc_synth", launch_b(MODE == MODE_TF32 ? Body::TcSynthTf32 : Body::TcSynthBf16,
                                        (int)tmem_cols_for(32 * g.chunk), 0, k_tc_synth<MODE>, dim3(p->R + 1, nchunks), dim3(kTcThreads), smem, st,
                                        s->map_syn, g));
    return MLSDC_OK;
}

// The warp-specialised analysis applies to latitude-contiguous launches of
// up to 8 members per CTA (two accumulator buffers of 2 x 16 x chunk
// columns in the 512 of tensor memory) without a fused node update.
inline bool ws_applies(const TcArgs& g) { return g.fo.sj == 1 && g.chunk <= 8; }
inline int cfg_index(int stage) { return stage == 0 ? 0 : 1; }

template <int MODE>
mlsdc_status launch_anal_ws(sh_plan_t p, TcState* s, const TcArgs& g, cudaStream_t st) {
    const int nchunks = (g.members + g.chunk - 1) / g.chunk;
    const size_t smem = cta_smem_bytes(MODE, g.chunk, g.stages);
    mlsdc_status rs = raise_smem_limit((const void*)k_tc_anal_ws<MODE>, smem);
    if (rs != MLSDC_OK) return rs;
    int per_sm = 0, sms = 0, dev = 0;
    MLSDC_CUDA(cudaGetDevice(&dev));
    MLSDC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MLSDC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_anal_ws<MODE>, kWsThreads, smem));
    // one wave of persistent CTAs, shared by the member chunks
    const int nx = std::min(s->n_tiles, std::max(1, per_sm * sms / nchunks));
    MLSDC_LAUNCH("k_tc_anal_ws",
                 launch_b(MODE == MODE_TF32 ? Body::TcAnalWsTf32 : Body::TcAnalWsBf16,
                                   (int)tmem_cols_for(64 * g.chunk), 0, k_tc_anal_ws<MODE>, dim3(nx, nchunks), dim3(kWsThreads), smem, st, s->map_ana, g));
    return MLSDC_OK;
}

template <int MODE>
mlsdc_status launch_anal(sh_plan_t p, TcState* s, const TcArgs& g, cudaStream_t st) {
    if (s->cfg[1].ws && ws_applies(g)) return launch_anal_ws<MODE>(p, s, g, st);
    const int nchunks = (g.members + g.chunk - 1) / g.chunk;
    const size_t smem = cta_smem_bytes(MODE, g.chunk, g.stages);
    mlsdc_status rs = raise_smem_limit((const void*)k_tc_anal<MODE>, smem);
    if (rs != MLSDC_OK) return rs;
    MLSDC_LAUNCH("k_tc_anal", launch_b(MODE == MODE_TF32 ? Body::TcAnalTf32 : Body::TcAnalBf16,
                                       (int)tmem_cols_for(32 * g.chunk), 0, k_tc_anal<MODE>, dim3(s->n_tiles, nchunks), dim3(kTcThreads), smem, st,
                                       s->map_ana, g));
    return MLSDC_OK;
}

// stage 0: the synthesis's configuration, 2: the analysis's
TcArgs base_args(sh_plan_t p, TcState* s, double a, int members, int stage) {
    const TcState::Cfg& cf = s->cfg[cfg_index(stage)];
    TcArgs g{};
    g.R = p->R;
    g.J2 = p->J2;
    g.nc = p->nc;
    g.J2p = s->J2p;
    g.members = members;
    g.chunk = std::min(cf.chunk, members);
    g.stages = cf.stages > 0 ? cf.stages : stages_for(s->mode, g.chunk);
    g.ia_f = (float)(1.0 / a);
    g.na2_f = (float)(-a * a);
    g.invnn = p->mp.invnn32;
    g.four_in = p->mp.four_in;
    g.four_out = p->mp.four_out;
    g.fo = four_out_layout(p->J, p->R, members >= kLatContigMembers);
    g.cor = p->d_cor;
    g.tiles = s->d_tiles;
    g.n_tiles = s->n_tiles;
    g.err = s->d_err;
    return g;
}

// Autotuner: for a full batch of members, time each Legendre stage that the
// plan's size rule runs on tensor cores at that batch (both when it runs
// neither, so a forced choice still gets a tuned configuration), on its own,
// with each feasible member chunk (1, 2, 4, 8, 16 members per CTA), K
// pipeline depth (two stages, or one, which leaves room for more CTAs per
// SM) and, for the analysis of batched launches, the warp-specialised
// kernel, and keep each stage's fastest.  Each candidate is timed inside a
// CUDA graph of kTuneReps launches (the launch cost of the step graphs, not
// the host's launch rate); a later candidate must win by 1 % to replace an
// earlier one, so near-ties do not flip between runs.  Runs once per plan,
// on zero inputs, at plan creation.
constexpr int kTuneReps = 10;
template <int MODE>
mlsdc_status autotune(sh_plan_t p, TcState* s) {
    const int B = p->max_members;
    bool syn = stage_uses_tc(p, 0, B), ana = stage_uses_tc(p, 2, B);
    if (!syn && !ana) syn = ana = true;
    const size_t n = (size_t)B * 3 * p->nc;
    double2 *x = nullptr, *fe = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&x, n * sizeof(double2)));
    MLSDC_CUDA(cudaMalloc((void**)&fe, n * sizeof(double2)));
    MLSDC_CUDA(cudaMemset(x, 0, n * sizeof(double2)));
    cudaStream_t st = nullptr;
    MLSDC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    mlsdc_status rs = MLSDC_OK;
    for (int stage = 0; stage <= 2 && rs == MLSDC_OK; stage += 2) {
        if (stage == 0 ? !syn : !ana) continue;
        TcState::Cfg& cf = s->cfg[cfg_index(stage)];
        TcState::Cfg best_cf = cf;
        float best = 1e30f;
        for (int k = 0; k < 20 && rs == MLSDC_OK; ++k) {
            // (chunk, stages, ws) = (1,1,0), (1,1,1), (1,2,0), (1,2,1), (2,1,0), ...
            const int chunk = 1 << (k >> 2), stages = 1 + ((k >> 1) & 1), ws = k & 1;
            if (chunk > B || cta_smem_bytes(MODE, chunk, stages) > kSmemBudget) continue;
            if (ws && !(stage == 2 && B >= kLatContigMembers && chunk <= 8)) continue;  // where the ws kernel applies
            cf.chunk = chunk;
            cf.stages = stages;
            cf.ws = ws;
            TcArgs g = base_args(p, s, 6.37122e6, B, stage);
            g.state = x;
            g.state_ms = (size_t)3 * p->nc;
            g.FE = fe;
            g.fe_ms = (size_t)3 * p->nc;
            auto enqueue = [&](cudaStream_t q) -> mlsdc_status {
                return stage == 0 ? launch_synth<MODE>(p, s, g, q) : launch_anal<MODE>(p, s, g, q);
            };
            rs = enqueue(st);  // outside the capture: sets the kernel's shared-memory limit
            if (rs == MLSDC_OK) MLSDC_CUDA(cudaStreamSynchronize(st));
            float ms = 0.f;
            if (rs == MLSDC_OK) rs = time_in_graph(st, kTuneReps, &ms, enqueue);
            if (rs == MLSDC_OK && ms < 0.99f * best) {
                best = ms;
                best_cf = cf;
            }
        }
        cf = best_cf;
    }
    cudaStreamDestroy(st);
    cudaFree(x);
    cudaFree(fe);
    return rs;
}

}  // namespace

bool make_rows_map_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                       uint32_t box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * sizeof(float)};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

mlsdc_status tc_init(sh_plan_t p) {
    if (p->J2 > kTileRows || p->R + 1 > kMaxKS) {
        set_error_text("tensor-core precisions need nlat/2 <= 128 and R <= 191");
        return MLSDC_ERR_INVALID;
    }
    TcState* s = new TcState();
    p->mp.tc = s;
    s->mode = p->precision == MLSDC_TF32 ? MODE_TF32 : MODE_BF16X3;
    s->KS = (p->R + 1 + 63) / 64 * 64;
    s->J2p = (p->J2 + 63) / 64 * 64;
    MLSDC_CUDA(cudaMalloc((void**)&s->d_err, sizeof(int)));
    MLSDC_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
    std::vector<int2> tiles;
    for (int m = 0; m <= p->R; ++m)
        for (int t = 0; t * kTileRows < p->R + 1 - m; ++t) tiles.push_back(make_int2(m, t));
    s->n_tiles = (int)tiles.size();
    MLSDC_CUDA(cudaMalloc((void**)&s->d_tiles, tiles.size() * sizeof(int2)));
    MLSDC_CUDA(cudaMemcpy(s->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
    mlsdc_status rs = s->mode == MODE_TF32 ? build_tables<MODE_TF32>(p, s) : build_tables<MODE_BF16X3>(p, s);
    if (rs != MLSDC_OK) return rs;
    rs = s->mode == MODE_TF32 ? autotune<MODE_TF32>(p, s) : autotune<MODE_BF16X3>(p, s);
    if (rs != MLSDC_OK) return rs;
    MLSDC_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
    return MLSDC_OK;
}

void tc_free(sh_plan_t p) {
    TcState* s = st_of(p);
    if (!s) return;
    for (int q = 0; q < 4; ++q) {
        cudaFree(s->syn[q]);
        cudaFree(s->ana[q]);
    }
    cudaFree(s->d_err);
    cudaFree(s->d_tiles);
    delete s;
    p->mp.tc = nullptr;
}

mlsdc_status tc_synth(sh_plan_t p, const double* state, double a, RhsBatch b, cudaStream_t st) {
    TcState* s = st_of(p);
    TcArgs g = base_args(p, s, a, b.members, 0);
    g.state = (const double2*)state;
    g.state_ms = b.state_ms;
    return s->mode == MODE_TF32 ? launch_synth<MODE_TF32>(p, s, g, st) : launch_synth<MODE_BF16X3>(p, s, g, st);
}

mlsdc_status tc_anal(sh_plan_t p, double a, double* FE, const double* state, double two_omega, RhsBatch b,
                     FourStride fo, cudaStream_t st) {
    TcState* s = st_of(p);
    TcArgs g = base_args(p, s, a, b.members, 2);
    g.state = (const double2*)state;
    g.state_ms = b.state_ms;
    g.two_omega = two_omega;
    g.FE = (double2*)FE;
    g.fe_ms = b.fe_ms;
    g.fo = fo;
    return s->mode == MODE_TF32 ? launch_anal<MODE_TF32>(p, s, g, st) : launch_anal<MODE_BF16X3>(p, s, g, st);
}

mlsdc_status tc_config(sh_plan_t p, int stage, int* chunk, int* stages, int* ws) {
    TcState* s = st_of(p);
    if (stage != 0 && stage != 2) return MLSDC_ERR_INVALID;
    const TcState::Cfg* cf = s ? &s->cfg[cfg_index(stage)] : nullptr;
    if (chunk) *chunk = cf ? cf->chunk : 0;
    if (stages) *stages = cf ? (cf->stages > 0 ? cf->stages : stages_for(s->mode, cf->chunk)) : 0;
    if (ws) *ws = cf ? cf->ws : 0;
    return MLSDC_OK;
}

mlsdc_status tc_set_config(sh_plan_t p, int stage, int chunk, int stages, int ws) {
    TcState* s = st_of(p);
    if (!s || (stage != 0 && stage != 2)) return MLSDC_ERR_INVALID;
    const bool pow2 = chunk >= 1 && chunk <= 16 && (chunk & (chunk - 1)) == 0;
    if (!pow2 || chunk > p->max_members || stages < 1 || stages > kMaxStages || ws < 0 || ws > 1 ||
        (ws && (stage == 0 || chunk > 8)) || cta_smem_bytes(s->mode, chunk, stages) > kSmemBudget)
        return MLSDC_ERR_INVALID;
    TcState::Cfg& cf = s->cfg[cfg_index(stage)];
    cf.chunk = chunk;
    cf.stages = stages;
    cf.ws = ws;
    return MLSDC_OK;
}

// One CTA waits on an mbarrier that nothing completes, with the kernels'
// bounded wait and a limit of limit_ns: the wait must give up and the kernel
// record kErrMmaTimeout and return (the check behind mlsdc_selftest_wait_timeout).
__global__ void k_wait_selftest(uint64_t limit_ns, int* code) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(sa(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) *code = mbar_wait(sa(&bar), 0, limit_ns) ? 0 : kErrMmaTimeout;
}

mlsdc_status wait_selftest(int timeout_ms, int* code) {
    int* d = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>((uint64_t)timeout_ms * 1000000ull, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(code, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_error("k_wait_selftest", e);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}

mlsdc_status tc_error(sh_plan_t p, int* code) {
    TcState* s = st_of(p);
    *code = 0;
    if (!s) return MLSDC_OK;
    MLSDC_CUDA(cudaMemcpy(code, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return MLSDC_OK;
}


}  // namespace mlsdc
