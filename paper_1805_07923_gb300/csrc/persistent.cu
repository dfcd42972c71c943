// The ensemble step (Algorithm 1 for every member of every truncation group,
// Sec. 4.3.2) as one persistent kernel launch.
//
// Each group's step is recorded, not launched: with a Recorder installed the
// step's launches (run_ops over build_mlsdc_ops) are stored as (body, grid,
// packed arguments), tagged with the step operation they belong to and their
// place within it.  The groups run the same operation list, so operation i of
// every group forms phase i (one phase per launch of an operation): the
// groups' launches of a phase are independent, and consecutive phases of one
// group depend on each other exactly as consecutive launches of its stream
// do.  The kernel runs the phases in order: each CTA takes work items of the
// phase (an item is `vpc` virtual blocks of one recorded launch, side by side
// on slices of the CTA's threads and shared memory, each with its own named
// barrier), runs the recorded body on them, and then meets every other CTA at
// a grid barrier before the next phase.  Every CTA must be resident for the
// barrier: the kernel is launched cooperatively, one CTA of 512 threads per
// SM (128 registers a thread: the register file of the SM).
//
// The grid barrier is a counter that each CTA's thread 0 increments with
// release semantics and polls with acquire semantics; the poll is bounded by
// the global timer (kBarrierNs) and an iteration cap.  A CTA whose wait gives
// up records kErrBarrierTimeout in the ensemble's error word, raises the
// kernel's abort flag and returns; every other CTA sees the flag in its own
// poll and returns too, so the launch ends (with the error readable through
// mlsdc_ensemble_device_error) instead of hanging.  The tensor-core bodies'
// own waits are bounded as in their kernels.
//
// Results are those of the graph of per-stage launches: the bodies are the
// kernels' code, run for the same blocks with the same arguments, and differ
// only where the compiler contracts an operation differently in the two
// compilations (split-BF16 ensembles: identical bit for bit, the float32
// epilogues round every operation explicitly; float64 ensembles: within
// 6e-16).
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "legendre_tc.cuh"
#include "rhs_kernels.cuh"
#include "sdc_internal.h"
#include "sdc_kernels.cuh"

namespace mlsdc {

Recorder*& active_recorder() {
    static thread_local Recorder* r = nullptr;
    return r;
}

namespace {

constexpr int kPThreads = 512;                     // threads per CTA of the persistent kernel
constexpr size_t kPSmem = 227 * 1024 - 1024;       // dynamic shared memory per CTA (bytes)
constexpr uint64_t kBarrierNs = 4000000000ull;     // a grid-barrier wait gives up after 4 s
constexpr uint32_t kBarrierSpins = 1u << 28;       // ... or after this many polls
constexpr int kErrBarrierTimeout = 3;              // (1 and 2 are the tensor-core kernels' codes)
constexpr unsigned kSlotBar0 = 2;                  // slot s: named barriers 2 + 2s and 3 + 2s
constexpr unsigned kMaxSlots = 7;                  // (16 named barriers per CTA)

// One recorded launch (a task).  Tasks are stored phase by phase, and within
// a phase the larger groups' first.
struct PRec {
    int body;                 // Body
    unsigned nt;              // threads per virtual block
    unsigned vpc;             // virtual blocks side by side per CTA
    unsigned gx, gy, gz;      // grid
    unsigned nblk;            // gx gy gz
    unsigned items;           // work items: ceil(nblk / vpc)
    unsigned item0;           // lockstep: the phase's first item of this task
    unsigned gitem0;          // dataflow: the step's first item of this task
    int dep;                  // dataflow: the same group's previous task (-1: none)
    unsigned smem;            // shared-memory slice per virtual block (bytes)
    unsigned long long args;  // byte offset of the packed arguments
};
struct PPhase {
    int r0, r1;      // records [r0, r1)
    unsigned items;  // work items of the phase
    int pad;
};
// The two schedules of the step's tasks:
//   lockstep: phase after phase, every CTA meeting the others at a grid
//     barrier between phases (the groups' launches of a phase side by side);
//   dataflow: one ticket counter hands out the work items of all tasks in
//     their stored order; a CTA that draws an item first waits until the
//     group's previous task has completed all its items (a per-task
//     completion counter), runs it, and counts it complete.  The groups move
//     through their phases independently, as the graph's per-group streams
//     do.  An item only waits on items with smaller tickets, which CTAs that
//     are running hold, so the schedule always progresses.
constexpr int kLockstep = 0, kDataflow = 1;

struct PArgs {
    const PPhase* phases;
    const PRec* recs;
    const unsigned char* argbuf;
    int nphases, nrecs, schedule;
    unsigned total_items;
    unsigned* bar;     // lockstep: arrivals so far            } zeroed before
    int* abort;        // raised by a CTA whose wait gave up    } each launch
    unsigned* ticket;  // dataflow: next item                   }
    unsigned* done;    // dataflow: completed items per task    }
    int* err;          // kErrBarrierTimeout when a wait gave up (sticky)
    uint64_t limit_ns;
    uint64_t* stamps;  // lockstep only: null, or [nphases + 1] timer readings of CTA 0 at the phase boundaries
};

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until *count reaches target (acquire), or give up (this
// thread's limit, recorded, or another CTA's abort).
__device__ bool wait_count(const unsigned* count, unsigned target, int* err, int* abort, uint64_t limit_ns) {
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0;; ++i) {
        if (ld_acquire(count) >= target) break;
        if (ld_relaxed(abort)) return false;
        if (((i & 15) == 15 && now_ns() - t0 > limit_ns) || i >= kBarrierSpins) {
            atomicExch(err, kErrBarrierTimeout);
            atomicExch(abort, 1);
            return false;
        }
        __nanosleep(32);
    }
    __threadfence();
    return true;
}

// Every CTA arrives; returns once `target` arrivals are counted, or false if
// the wait gave up (this CTA's limit, or another CTA's abort).
__device__ bool grid_barrier(unsigned* count, unsigned target, int* err, int* abort, uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();  // the CTA's work of the phase is done
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_add(count, 1);
        s_ok = wait_count(count, target, err, abort, limit_ns) ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}

#define MLSDC_STRIP_(...) __VA_ARGS__
#define MLSDC_STRIP(x) MLSDC_STRIP_ x
// case: run body BODY on the pack at `a` (the pack of BODY's parameters)
#define MLSDC_BODY_CASE(ID, BODY)                                                                   \
    case Body::ID: {                                                                                \
        auto f = [](const Blk& bb, const auto&... x) { MLSDC_STRIP(BODY)(bb, x...); };              \
        apply_pack(f, b, *reinterpret_cast<const typename BodyPack<decltype(&MLSDC_STRIP(BODY))>::type*>(a)); \
        break;                                                                                      \
    }

__device__ __forceinline__ void run_body(int body, const Blk& b, const unsigned char* a) {
    switch ((Body)body) {
        MLSDC_BODY_CASE(SynthF32, (b_synth_rhs<float, false>))
        MLSDC_BODY_CASE(SynthF32Tma, (b_synth_rhs<float, true>))
        MLSDC_BODY_CASE(SynthF64, (b_synth_rhs<double, false>))
        MLSDC_BODY_CASE(GridF32x1, (b_grid_rhs<float, 1>))
        MLSDC_BODY_CASE(GridF32x2, (b_grid_rhs<float, 2>))
        MLSDC_BODY_CASE(GridF64x1, (b_grid_rhs<double, 1>))
        MLSDC_BODY_CASE(AnalF32, (b_anal_rhs<float>))
        MLSDC_BODY_CASE(AnalF64, (b_anal_rhs<double>))
        MLSDC_BODY_CASE(TcSynthTf32, (tc::b_tc_synth<tc::MODE_TF32>))
        MLSDC_BODY_CASE(TcSynthBf16, (tc::b_tc_synth<tc::MODE_BF16X3>))
        MLSDC_BODY_CASE(TcAnalTf32, (tc::b_tc_anal<tc::MODE_TF32>))
        MLSDC_BODY_CASE(TcAnalBf16, (tc::b_tc_anal<tc::MODE_BF16X3>))
        MLSDC_BODY_CASE(TcAnalWsTf32, (tc::b_tc_anal_ws<tc::MODE_TF32>))
        MLSDC_BODY_CASE(TcAnalWsBf16, (tc::b_tc_anal_ws<tc::MODE_BF16X3>))
        MLSDC_BODY_CASE(ImplicitRhs, (b_implicit_rhs))
        MLSDC_BODY_CASE(SweepNode, (b_sweep_node))
        MLSDC_BODY_CASE(SweepNode0_2, (b_sweep_node0<2>))
        MLSDC_BODY_CASE(SweepNode0_3, (b_sweep_node0<3>))
        MLSDC_BODY_CASE(SweepNode0_4, (b_sweep_node0<4>))
        MLSDC_BODY_CASE(SweepNode0_5, (b_sweep_node0<5>))
        MLSDC_BODY_CASE(SweepNode0_6, (b_sweep_node0<6>))
        MLSDC_BODY_CASE(SweepNode0_7, (b_sweep_node0<7>))
        MLSDC_BODY_CASE(SweepNode0_8, (b_sweep_node0<8>))
        MLSDC_BODY_CASE(SweepNodeS, (b_sweep_node_s))
        MLSDC_BODY_CASE(Broadcast, (b_broadcast))
        MLSDC_BODY_CASE(Restrict, (b_restrict))
        MLSDC_BODY_CASE(FasTau, (b_fas_tau))
        MLSDC_BODY_CASE(Interp, (b_interp))
        MLSDC_BODY_CASE(PadAdd, (b_pad_add))
        MLSDC_BODY_CASE(Copy2D, (b_copy2d))
        default:
            break;
    }
}

// Item `item` of task R: vpc virtual blocks side by side, then the CTA's
// barrier (every thread of the CTA calls this).
__device__ __forceinline__ void run_item(const PArgs& a, const PRec& R, unsigned item, unsigned char* smem_p) {
    const unsigned slot = threadIdx.x / R.nt;
    const unsigned vb = item * R.vpc + slot;
    if (slot < R.vpc && vb < R.nblk) {
        Blk b;
        b.idx = make_uint3(vb % R.gx, (vb / R.gx) % R.gy, vb / (R.gx * R.gy));
        b.dim = make_uint3(R.gx, R.gy, R.gz);
        b.t = threadIdx.x - slot * R.nt;
        b.nt = R.nt;
        b.bar = R.nt == kPThreads ? 0u : kSlotBar0 + 2 * slot;
        b.bar2 = kSlotBar0 + 2 * slot + 1;
        b.smem = smem_p + (size_t)slot * R.smem;
        b.persist = true;
        run_body(R.body, b, a.argbuf + R.args);
    }
    // the next item's bodies may hand this shared memory to TMA or the
    // tensor cores (async proxy): order this thread's accesses first
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
}

__global__ void __launch_bounds__(kPThreads, 1) k_persistent(const __grid_constant__ PArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_p[];
    if (a.schedule == kDataflow) {
        __shared__ int s_r;
        __shared__ unsigned s_item;
        int r_cur = 0;  // thread 0: this CTA's tickets only grow, so the task search moves forward
        for (;;) {
            if (threadIdx.x == 0) {
                int r = -1;
                unsigned item = 0;
                const unsigned t = atomicAdd(a.ticket, 1u);
                if (t < a.total_items && !ld_relaxed(a.abort)) {
                    while (r_cur + 1 < a.nrecs && t >= a.recs[r_cur + 1].gitem0) ++r_cur;
                    r = r_cur;
                    item = t - a.recs[r].gitem0;
                    const int dep = a.recs[r].dep;
                    if (dep >= 0 && !wait_count(a.done + dep, a.recs[dep].items, a.err, a.abort, a.limit_ns)) r = -1;
                }
                s_r = r;
                s_item = item;
            }
            __syncthreads();
            const int r = s_r;
            if (r < 0) break;
            run_item(a, a.recs[r], s_item, smem_p);
            if (threadIdx.x == 0) {
                __threadfence();
                red_release_add(a.done + r, 1);
            }
        }
        return;
    }
    if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0) a.stamps[0] = now_ns();
    for (int ph = 0; ph < a.nphases; ++ph) {
        const PPhase P = a.phases[ph];
        for (unsigned it = blockIdx.x; it < P.items; it += gridDim.x) {
            int r = P.r0;
            while (r + 1 < P.r1 && it >= a.recs[r + 1].item0) ++r;
            run_item(a, a.recs[r], it - a.recs[r].item0, smem_p);
        }
        if (ph + 1 < a.nphases &&
            !grid_barrier(a.bar, (unsigned)(ph + 1) * gridDim.x, a.err, a.abort, a.limit_ns))
            return;
        if (a.stamps && blockIdx.x == 0 && threadIdx.x == 0) a.stamps[ph + 1] = now_ns();
    }
}

// Two CTAs wait on a barrier that expects one arrival more than the grid
// has: both waits must give up after limit_ns (mlsdc_selftest_grid_barrier_timeout).
__global__ void k_barrier_selftest(unsigned* count, int* err, int* abort, uint64_t limit_ns) {
    grid_barrier(count, gridDim.x + 1, err, abort, limit_ns);
}

// The recorded form of one ensemble step (one per states, dt, n_iter, n_c).
struct PStep {
    int schedule = kLockstep;
    std::vector<PPhase> phases;
    std::vector<PRec> recs;
    std::vector<unsigned char> args;
    unsigned total_items = 0;
    PPhase* d_phases = nullptr;
    PRec* d_recs = nullptr;
    unsigned char* d_args = nullptr;
    unsigned* d_sync = nullptr;       // [0] barrier, [1] abort, [2] ticket, [3] unused, [4..) completed items per task
    cudaGraphExec_t graph = nullptr;  // the reset and the kernel (null: launched directly)
};
struct PState {
    std::map<std::tuple<std::vector<double*>, double, int, int, int>, PStep*> steps;
    int* d_err = nullptr;
    int ctas = 0;
    int schedule = kLockstep;  // measured faster than the dataflow schedule on the 96-member ensemble
    PStep* last = nullptr;
};

void free_step(PStep* s) {
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    cudaFree(s->d_phases);
    cudaFree(s->d_recs);
    cudaFree(s->d_args);
    cudaFree(s->d_sync);
    delete s;
}

mlsdc_status pstate_of(mlsdc_ensemble_t e, PState** out) {
    if (!e->persist) {
        PState* ps = new PState();
        e->persist = ps;
        MLSDC_CUDA(cudaMalloc((void**)&ps->d_err, sizeof(int)));
        MLSDC_CUDA(cudaMemset(ps->d_err, 0, sizeof(int)));
        MLSDC_CUDA(cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem));
        int dev = 0, sms = 0, per_sm = 0;
        MLSDC_CUDA(cudaGetDevice(&dev));
        MLSDC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MLSDC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, kPThreads, kPSmem));
        if (per_sm < 1) return invalid_arg("persistent ensemble kernel: no CTA fits an SM");
        ps->ctas = sms * per_sm;
    }
    *out = reinterpret_cast<PState*>(e->persist);
    return MLSDC_OK;
}

// Record every group's step and lay the launches out as phases.
mlsdc_status build_step(mlsdc_ensemble_t e, const std::vector<double*>& states, double dt, int n_iter, int n_c,
                        PStep* ps) {
    std::vector<std::vector<RecLaunch>> per_group;
    for (size_t g = 0; g < e->groups.size(); ++g) {
        mlsdc_t ml = e->groups[g];
        if ((ml->f->options | ml->c->options) & MLSDC_CORIOLIS_IMPLICIT)
            return invalid_arg("persistent ensemble step: implicit-Coriolis levels are not supported");
        Recorder rec;
        active_recorder() = &rec;
        std::vector<Op> ops;
        ml->f->cur = ml->c->cur = 0;
        build_mlsdc_ops(ml, (double2*)states[g], dt, n_iter, n_c, ops);
        int64_t launches = 0;
        const mlsdc_status s = run_ops(ml, ops, nullptr, &launches, nullptr);
        active_recorder() = nullptr;
        ml->f->cur = ml->c->cur = 0;
        if (rec.refused) return invalid_arg("persistent ensemble step: an operation of the step has no device body");
        if (s != MLSDC_OK) return s;
        per_group.push_back(std::move(rec.recs));
    }
    // phase key (operation, place within it) -> the groups' launches
    std::map<std::pair<int, int>, std::vector<const RecLaunch*>> by_key;
    for (const auto& recs : per_group)
        for (const RecLaunch& r : recs) by_key[{r.op, r.sub}].push_back(&r);
    std::map<const RecLaunch*, int> group_of;
    for (size_t g = 0; g < per_group.size(); ++g)
        for (const RecLaunch& r : per_group[g]) group_of[&r] = (int)g;
    std::vector<int> last_task(per_group.size(), -1);
    for (auto& kv : by_key) {
        PPhase P{};
        P.r0 = (int)ps->recs.size();
        unsigned items = 0;
        // the larger launches of the phase first (the dataflow schedule hands them out first)
        std::stable_sort(kv.second.begin(), kv.second.end(), [](const RecLaunch* x, const RecLaunch* y) {
            return (size_t)x->grid.x * x->grid.y * x->grid.z > (size_t)y->grid.x * y->grid.y * y->grid.z;
        });
        for (const RecLaunch* r : kv.second) {
            if (r->block.y != 1 || r->block.z != 1 || r->block.x % 32 || r->block.x > (unsigned)kPThreads)
                return invalid_arg("persistent ensemble step: a launch's block shape does not fit the kernel");
            PRec R{};
            R.body = (int)r->body;
            R.nt = r->block.x;
            R.smem = (unsigned)((r->smem + 127) / 128 * 128);
            unsigned vpc = std::min<unsigned>(kPThreads / R.nt, kMaxSlots);
            if (R.smem) vpc = std::min<unsigned>(vpc, (unsigned)(kPSmem / R.smem));
            if (r->tmem_cols) vpc = std::min<unsigned>(vpc, 512u / (unsigned)r->tmem_cols);
            if (vpc < 1) return invalid_arg("persistent ensemble step: a launch needs more shared memory than a CTA has");
            R.vpc = vpc;
            R.gx = r->grid.x;
            R.gy = r->grid.y;
            R.gz = r->grid.z;
            R.nblk = R.gx * R.gy * R.gz;
            R.items = (R.nblk + vpc - 1) / vpc;
            R.item0 = items;
            items += R.items;
            R.gitem0 = ps->total_items;
            ps->total_items += R.items;
            const int g = group_of[r];
            R.dep = last_task[g];
            last_task[g] = (int)ps->recs.size();
            size_t off = (ps->args.size() + 127) / 128 * 128;
            ps->args.resize(off + r->args.size());
            std::memcpy(ps->args.data() + off, r->args.data(), r->args.size());
            R.args = off;
            ps->recs.push_back(R);
        }
        P.r1 = (int)ps->recs.size();
        P.items = items;
        ps->phases.push_back(P);
    }
    MLSDC_CUDA(cudaMalloc((void**)&ps->d_phases, ps->phases.size() * sizeof(PPhase)));
    MLSDC_CUDA(cudaMalloc((void**)&ps->d_recs, ps->recs.size() * sizeof(PRec)));
    MLSDC_CUDA(cudaMalloc((void**)&ps->d_args, std::max<size_t>(ps->args.size(), 128)));
    MLSDC_CUDA(cudaMemcpy(ps->d_phases, ps->phases.data(), ps->phases.size() * sizeof(PPhase),
                          cudaMemcpyHostToDevice));
    MLSDC_CUDA(cudaMemcpy(ps->d_recs, ps->recs.data(), ps->recs.size() * sizeof(PRec), cudaMemcpyHostToDevice));
    MLSDC_CUDA(cudaMemcpy(ps->d_args, ps->args.data(), ps->args.size(), cudaMemcpyHostToDevice));
    MLSDC_CUDA(cudaMalloc((void**)&ps->d_sync, (4 + ps->recs.size()) * sizeof(unsigned)));
    return MLSDC_OK;
}

// The two resets and the cooperative launch of one step.
mlsdc_status enqueue_step(const PState* st, const PStep* ps, cudaStream_t s, uint64_t* stamps = nullptr) {
    MLSDC_CUDA(cudaMemsetAsync(ps->d_sync, 0, (4 + ps->recs.size()) * sizeof(unsigned), s));
    PArgs a;
    a.phases = ps->d_phases;
    a.recs = ps->d_recs;
    a.argbuf = ps->d_args;
    a.nphases = (int)ps->phases.size();
    a.nrecs = (int)ps->recs.size();
    a.schedule = ps->schedule;
    a.total_items = ps->total_items;
    a.bar = ps->d_sync;
    a.abort = reinterpret_cast<int*>(ps->d_sync + 1);
    a.ticket = ps->d_sync + 2;
    a.done = ps->d_sync + 4;
    a.err = st->d_err;
    a.limit_ns = kBarrierNs;
    a.stamps = stamps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(st->ctas);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = kPSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MLSDC_CUDA(cudaLaunchKernelEx(&cfg, k_persistent, a));
    return MLSDC_OK;
}

}  // namespace

void persistent_free(mlsdc_ensemble_t e) {
    PState* st = reinterpret_cast<PState*>(e->persist);
    if (!st) return;
    for (auto& kv : st->steps) free_step(kv.second);
    cudaFree(st->d_err);
    delete st;
    e->persist = nullptr;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status mlsdc_ensemble_step_persistent(mlsdc_ensemble_t e, double* const* states, double dt,
                                                       int n_iter, int n_coarse_sweeps, void* stream) {
    if (!e || !states || n_iter < 0 || n_coarse_sweeps < 0) return MLSDC_ERR_INVALID;
    std::vector<double*> sv(states, states + e->groups.size());
    for (double* p : sv) {
        if (!p) return MLSDC_ERR_INVALID;
        MLSDC_ALIGNED("mlsdc_ensemble_step_persistent", {"states[i]", p});
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (mlsdc_t ml : e->groups) {
        mlsdc_status sp = prepare_levels(ml, dt, st);
        if (sp != MLSDC_OK) return sp;
    }
    PState* ps = nullptr;
    mlsdc_status s = pstate_of(e, &ps);
    if (s != MLSDC_OK) return s;
    auto key = std::make_tuple(sv, dt, n_iter, n_coarse_sweeps, ps->schedule);
    auto it = ps->steps.find(key);
    if (it == ps->steps.end()) {
        PStep* step = new PStep();
        step->schedule = ps->schedule;
        s = build_step(e, sv, dt, n_iter, n_coarse_sweeps, step);
        if (s != MLSDC_OK) {
            free_step(step);
            return s;
        }
        // capture the resets and the launch once; a stream that cannot
        // capture the cooperative launch keeps direct launches
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        bool captured = cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (captured) {
            const mlsdc_status se = enqueue_step(ps, step, e->cap);
            captured = cudaStreamEndCapture(e->cap, &g) == cudaSuccess && se == MLSDC_OK && g &&
                       cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!captured) {
            if (ex) cudaGraphExecDestroy(ex);
            ex = nullptr;
            cudaGetLastError();
        }
        step->graph = ex;
        it = ps->steps.emplace(key, step).first;
    }
    ps->last = it->second;
    e->launches = 1;  // one kernel per step (and two 4-byte memsets)
    if (it->second->graph) {
        MLSDC_CUDA(cudaGraphLaunch(it->second->graph, st));
        return MLSDC_OK;
    }
    return enqueue_step(ps, it->second, st);
}

extern "C" mlsdc_status mlsdc_ensemble_persistent_schedule(mlsdc_ensemble_t e, int schedule) {
    if (!e || (schedule != kLockstep && schedule != kDataflow)) return MLSDC_ERR_INVALID;
    PState* ps = nullptr;
    mlsdc_status s = pstate_of(e, &ps);
    if (s != MLSDC_OK) return s;
    ps->schedule = schedule;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_ensemble_persistent_info(mlsdc_ensemble_t e, int* phases, int* records, int* ctas,
                                                       int* in_graph) {
    if (!e || !e->persist) return MLSDC_ERR_INVALID;
    const PState* ps = reinterpret_cast<const PState*>(e->persist);
    if (!ps->last) return MLSDC_ERR_INVALID;
    if (phases) *phases = (int)ps->last->phases.size();
    if (records) *records = (int)ps->last->recs.size();
    if (ctas) *ctas = ps->ctas;
    if (in_graph) *in_graph = ps->last->graph ? 1 : 0;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_ensemble_device_error(mlsdc_ensemble_t e, int* code) {
    if (!e || !code) return MLSDC_ERR_INVALID;
    *code = 0;
    const PState* ps = reinterpret_cast<const PState*>(e->persist);
    if (!ps) return MLSDC_OK;
    MLSDC_CUDA(cudaMemcpy(code, ps->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_selftest_grid_barrier_timeout(int timeout_ms, int* code) {
    if (!code || timeout_ms < 1 || timeout_ms > 2000) return MLSDC_ERR_INVALID;
    unsigned* d = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&d, 16));
    cudaError_t err = cudaMemset(d, 0, 16);
    int* ip = reinterpret_cast<int*>(d);
    if (err == cudaSuccess) {
        k_barrier_selftest<<<2, 32>>>(d, ip + 1, ip + 2, (uint64_t)timeout_ms * 1000000ull);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpy(code, ip + 1, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) {
        set_error("k_barrier_selftest", err);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_ensemble_persistent_phase_times(mlsdc_ensemble_t e, float* phase_us, int* phase_body,
                                                              int cap, void* stream) {
    if (!e || !e->persist || !phase_us || !phase_body || cap < 1) return MLSDC_ERR_INVALID;
    const PState* ps = reinterpret_cast<const PState*>(e->persist);
    const PStep* step = ps->last;
    if (!step) return MLSDC_ERR_INVALID;
    if (step->schedule != kLockstep)
        return invalid_arg("mlsdc_ensemble_persistent_phase_times: phases are timed under the lockstep schedule");
    const int np = (int)step->phases.size();
    if (cap < np) return invalid_arg("mlsdc_ensemble_persistent_phase_times: room for fewer phases than the step has");
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* d = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&d, (size_t)(np + 1) * sizeof(uint64_t)));
    std::vector<uint64_t> h(np + 1, 0);
    mlsdc_status s = enqueue_step(ps, step, st, d);
    cudaError_t err = s == MLSDC_OK ? cudaStreamSynchronize(st) : cudaSuccess;
    if (s == MLSDC_OK && err == cudaSuccess)
        err = cudaMemcpy(h.data(), d, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (s != MLSDC_OK) return s;
    if (err != cudaSuccess) {
        set_error("mlsdc_ensemble_persistent_phase_times", err);
        return MLSDC_ERR_CUDA;
    }
    for (int p = 0; p < np; ++p) {
        phase_us[p] = (float)((double)(h[p + 1] - h[p]) * 1e-3);
        // the body of the phase's record with the most blocks
        int best = step->phases[p].r0;
        for (int r = step->phases[p].r0; r < step->phases[p].r1; ++r)
            if (step->recs[r].nblk > step->recs[best].nblk) best = r;
        phase_body[p] = step->recs[best].body;
    }
    return MLSDC_OK;
}
