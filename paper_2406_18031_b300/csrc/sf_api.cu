// sf_api.cu -- host side of libsf: filter engines, launch plans and the C ABI
// of include/sf.h.  All device work is issued on the caller's stream (and, for
// sf_submit_host, the context's two copy streams); nothing here synchronises
// except sf_status / sf_batch_status, sf_step_host, sf_wait_host, creation
// (and its autotuner) and the stage entry points' descriptor uploads.
//
// An engine is a set of independent camera streams, each with its pyramid
// levels.  Its frame is a fixed sequence of launches whose descriptors are
// built once: the propagation launches (every level of every stream), one
// solve launch (every level), then the smoothing + reconstruction cascade
// (one launch per pyramid depth, top levels first; or one smoothing launch and
// light reconstruction launches, update mode 2).  sf_ctx is an engine of
// one stream fed through per-frame pointers; sf_batch is an engine of many
// streams with library-owned input/output slots, replayed from CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <random>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sf.h"
#include "sf_conv.cuh"
#include "sf_kernels.cuh"
#include "sf_surrogate.cuh"

using namespace sfdev;

namespace {

// the largest number of sub-iterations fused in one propagation launch (its
// square output tile is 64 - 2 nf pixels wide); an engine may use fewer
constexpr int kNfLimit = 8;

// the largest frame (pixels): plane offsets of the kernels are 32-bit, and a
// frame of this size already needs 137 GB of state
constexpr long long kMaxPixels = 1LL << 30;

// streaming multiprocessors of a B300 (two dies of 74): grid sizes of the
// grid-stride kernels and the launch-form thresholds are multiples of it
constexpr int kSmCount = 148;

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

Grid make_grid(const sf_grid& s)
{
    Grid g;
    g.H = s.H;
    g.W = s.W;
    g.ax = 1.0f / s.fx;
    g.bx = (0.5f - s.cx) / s.fx;
    g.ay = 1.0f / s.fy;
    g.by = (0.5f - s.cy) / s.fy;
    g.a = 1.0f / s.fx;
    return g;
}

// the dynamic shared-memory limit of a kernel, raised once per device and size
// (so that launches inside a graph capture never need the attribute call)
int set_smem_attr(const void* fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return SF_OK;
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, const void*>, size_t>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SF_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : done)
        if (e.first.first == dev && e.first.second == fn && e.second >= bytes) return SF_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return SF_ECUDA;
    done.push_back({{dev, fn}, bytes});
    return SF_OK;
}

int last_error() { return cudaGetLastError() == cudaSuccess ? SF_OK : SF_ECUDA; }

// NVTX range around the host-side issue of one stage's launch (visible in a
// system trace next to the kernel it issued).  Off unless sf_set_trace(1):
// with a tracing tool injected a range costs microseconds of host time, which
// a 60-microsecond frame cannot hide.
std::atomic<int> g_trace{0};

struct NvtxRange {
    const bool on;
    explicit NvtxRange(const char* name) : on(g_trace.load(std::memory_order_relaxed) != 0)
    {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxRange()
    {
        if (on) nvtxRangePop();
    }
};

// The frame's kernels are launched with programmatic stream serialisation:
// each may be scheduled while the previous kernel of the stream finishes, and
// waits (pdl_wait) before it touches anything that kernel or earlier work
// produced, so only launch latency and index set-up overlap.
//
// Rule for every caller: the kernels read their launch descriptors (jobs and
// work items) BEFORE pdl_wait, so a programmatic launch is correct only when
// those descriptors were written by no kernel of the stream (host uploads at
// plan creation).  A path whose descriptors come from a device kernel just
// before the launch must pass pdl = false (an ordinary, fully serialised
// launch), as sf_propagate_noalloc does.
constexpr bool kUsePdl = true;

template <typename... KArgs, typename... Args>
int launch_ex(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (kUsePdl && pdl) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...) == cudaSuccess ? SF_OK : SF_ECUDA;
}

template <typename... KArgs, typename... Args>
int launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    return launch_ex(true, kernel, grid, block, smem, st, args...);
}

// A launch: device copies of its jobs and of its work list (one item per CTA).
struct Plan {
    void* jobs = nullptr;
    int4* work = nullptr;
    int nwork = 0;
    size_t smem = 0;
    bool c8 = false;     // propagation: some job transports 8 channels
    int nf = 0;          // propagation: sub-iterations of the launch's longest job
    int warps = 16;      // propagation: warps per CTA (prop_warps of nf)
    bool resid = false;  // propagation: residual mode (k_propagate's RES form, 8 warps)
    int tile = 0;        // solve: tile edge (kSolveTSmall, else kSolveT)
};

template <class Job>
int upload_plan(const std::vector<Job>& jobs, const std::vector<int4>& work, Plan& p, cudaStream_t st)
{
    p.nwork = (int)work.size();
    if (jobs.empty()) return SF_OK;
    if (cudaMalloc(&p.jobs, jobs.size() * sizeof(Job)) != cudaSuccess) { p.jobs = nullptr; return SF_ENOMEM; }
    if (cudaMalloc(&p.work, work.size() * sizeof(int4)) != cudaSuccess) { p.work = nullptr; return SF_ENOMEM; }
    if (cudaMemcpyAsync(p.jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SF_ECUDA;
    if (cudaMemcpyAsync(p.work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SF_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
}

void free_plan(Plan& p)
{
    cudaFree(p.jobs);
    cudaFree(p.work);
    p = Plan();
}

void add_tiles(std::vector<int4>& work, int job, int H, int W, int TX, int TY)
{
    for (int ty = 0; ty < H; ty += TY)
        for (int tx = 0; tx < W; tx += TX) work.push_back(make_int4(job, ty, tx, 0));
}

// offset of the work list behind a job in one stage-call upload: int4 loads
// need 16-byte alignment whatever the size of the job struct
inline size_t work_offset(size_t job_bytes) { return (job_bytes + 255) & ~(size_t)255; }

template <bool C8, bool LIT, bool IMU, bool PE, int WARPS, bool RES = false>
int launch_propagate_t(const Plan& p, int parity, float wscale, int flags, int* status, float mscale, cudaStream_t st,
                       bool pdl)
{
    auto* kern = k_propagate<C8, LIT, IMU, PE, WARPS, RES>;
    if (set_smem_attr((const void*)kern, p.smem)) return SF_ECUDA;
    return launch_ex(pdl, kern, dim3(p.nwork), dim3(32 * WARPS), p.smem, st, (const PropJob*)p.jobs,
                     (const int4*)p.work, parity, wscale, flags, status, mscale);
}

template <bool C8, bool LIT, bool IMU>
int launch_propagate_i(const Plan& p, int parity, float wscale, int flags, int* status, float mscale, cudaStream_t st,
                       bool pdl)
{
    // 8-warp CTAs for launches of few sub-iterations (prop_warps); the padded
    // form for launches of many (see kPrPaddedNf)
    if (p.resid)   // the surrogate's check: one sub-iteration of top levels, 8-warp CTAs
        return p.warps == 8 && !C8 ? launch_propagate_t<false, LIT, IMU, false, 8, true>(p, parity, wscale, flags, status,
                                                                                          mscale, st, pdl)
                                   : SF_EINVAL;
    if (p.warps == 8)
        return launch_propagate_t<C8, LIT, IMU, false, 8>(p, parity, wscale, flags, status, mscale, st, pdl);
    if (p.nf >= kPrPaddedNf)
        return launch_propagate_t<C8, LIT, IMU, true, 16>(p, parity, wscale, flags, status, mscale, st, pdl);
    return launch_propagate_t<C8, LIT, IMU, false, 16>(p, parity, wscale, flags, status, mscale, st, pdl);
}

template <bool C8, bool LIT>
int launch_propagate_l(const Plan& p, int parity, float wscale, int flags, int* status, float mscale, cudaStream_t st,
                       bool pdl)
{
    if (flags & SF_IMU) return launch_propagate_i<C8, LIT, true>(p, parity, wscale, flags, status, mscale, st, pdl);
    return launch_propagate_i<C8, LIT, false>(p, parity, wscale, flags, status, mscale, st, pdl);
}

// one propagation launch; with SF_IMU in flags the jobs' motion slots hold
// (Omega, a) and mscale converts them to frame units (Omega mscale,
// a mscale^2): the frame time in seconds, or 1 for values already per frame.
// pdl = false for a plan whose descriptors a kernel has just written (see
// launch_ex).
int launch_propagate(const Plan& p, int parity, float wscale, int flags, int* status, cudaStream_t st,
                     float mscale = 1.0f, bool pdl = true)
{
    if (p.nwork == 0) return SF_OK;
    const bool lit = (flags & SF_DOMINANT_LITERAL) != 0;
    if (p.c8) return lit ? launch_propagate_l<true, true>(p, parity, wscale, flags, status, mscale, st, pdl)
                         : launch_propagate_l<true, false>(p, parity, wscale, flags, status, mscale, st, pdl);
    return lit ? launch_propagate_l<false, true>(p, parity, wscale, flags, status, mscale, st, pdl)
               : launch_propagate_l<false, false>(p, parity, wscale, flags, status, mscale, st, pdl);
}

int launch_solve(const Plan& p, const UpdArgs& a, cudaStream_t st)
{
    if (p.nwork == 0) return SF_OK;
    auto* kern = p.tile == kSolveTSmall ? k_solve<kSolveTSmall> : k_solve<kSolveT>;
    return launch_pdl(kern, dim3(p.nwork), dim3(kSolveThreads), 0, st, (const SolveJob*)p.jobs, (const int4*)p.work, a);
}

int launch_smooth(const Plan& p, int q, float inv_dt, int check_finite, int* status, float* flow, float* inv,
                  cudaStream_t st)
{
    if (p.nwork == 0) return SF_OK;
    // more than four CTAs per SM of work: the 4-CTA-per-SM form (see k_smooth_recon)
    auto* kern = p.nwork > 4 * kSmCount ? k_smooth_recon<4> : k_smooth_recon<3>;
    if (set_smem_attr((const void*)kern, p.smem)) return SF_ECUDA;
    return launch_pdl(kern, dim3(p.nwork), dim3(kSmoothThreads), p.smem, st, (const SmoothJob*)p.jobs,
                      (const int4*)p.work, q, inv_dt, check_finite, status, flow, inv);
}

int launch_recon(const Plan& p, int q, float inv_dt, int check_finite, int* status, float* flow, float* inv,
                 cudaStream_t st)
{
    if (p.nwork == 0) return SF_OK;
    return launch_pdl(k_recon_jobs, dim3(p.nwork), dim3(kThreads), 0, st, (const ReconJob*)p.jobs, (const int4*)p.work,
                      q, inv_dt, check_finite, status, flow, inv);
}

int launch_reconstruct(const ReconArgs& a, cudaStream_t st)
{
    const int n = a.H * a.W;
    const int blocks = std::min(ceil_div(n, kThreads), kSmCount * 8);
    k_reconstruct<<<blocks, kThreads, 0, st>>>(a);
    return last_error();
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// parameter checks shared by sf_create and sf_batch_create (no device calls)
int check_params(int H, int W, int L, const sf_params* p)
{
    if (!p || L < 1 || L > SF_MAX_LEVELS || L > kMaxLevelsDev) return SF_EINVAL;
    const int m = 1 << (L - 1);
    if (H <= 0 || W <= 0 || H % m || W % m || H / m < 8 || W / m < 8) return SF_EINVAL;
    if ((long long)H * W > kMaxPixels) return SF_EINVAL;
    if (!(p->fx > 0 && p->fy > 0) || !std::isfinite(p->fx) || !std::isfinite(p->fy) || !std::isfinite(p->cx) ||
        !std::isfinite(p->cy))
        return SF_EINVAL;
    if (!(p->lambda_ref > 0) || !std::isfinite(p->lambda_ref) || !(p->gamma[2] > 0) || !(p->gamma[4] > 0))
        return SF_EINVAL;
    for (int k = 0; k < 5; ++k)
        if (!(p->gamma[k] >= 0) || !std::isfinite(p->gamma[k])) return SF_EINVAL;
    if (!(p->max_flow >= 0) || !std::isfinite(p->max_flow)) return SF_EINVAL;
    if (p->nf_max < 0 || p->nf_max > kNfLimit) return SF_EINVAL;
    if (p->update_mode < 0 || p->update_mode > 2) return SF_EINVAL;
    if (p->solve_tile != 0 && p->solve_tile != kSolveTSmall && p->solve_tile != kSolveT) return SF_EINVAL;
    for (int h = 0; h < L; ++h) {
        const int N = p->iters[h] > 0 ? p->iters[h] : std::max(1, (int)std::ceil(p->max_flow / (float)(1 << h)));
        if (N > 4096 || p->smooth_iters[h] < 0 || p->smooth_iters[h] > 16) return SF_EINVAL;
    }
    return SF_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// per-launch timing
// ----------------------------------------------------------------------------

struct Profiler {
    int enabled = 0;
    std::vector<cudaEvent_t> pool;   // pairs, reused after a read
    std::vector<int> slot;           // launch slot of each recorded pair
    size_t used = 0;
    ~Profiler()
    {
        for (auto e : pool) cudaEventDestroy(e);
    }
    int read(float* ms, int* count, int n)
    {
        for (int k = 0; k < n; ++k) { ms[k] = 0.0f; count[k] = 0; }
        for (size_t p = 0; p < used; ++p) {
            if (cudaEventSynchronize(pool[2 * p + 1]) != cudaSuccess) return SF_ECUDA;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, pool[2 * p], pool[2 * p + 1]) != cudaSuccess) return SF_ECUDA;
            if (slot[p] < n) { ms[slot[p]] += t; count[slot[p]] += 1; }
        }
        used = 0;
        return SF_OK;
    }
};

// event pair around one launch of slot `slot` (no-op unless profiling)
struct ProfScope {
    Profiler& pr;
    cudaStream_t st;
    size_t pair;
    ProfScope(Profiler& p, int slot_, cudaStream_t st_) : pr(p), st(st_), pair((size_t)-1)
    {
        if (!pr.enabled) return;
        if (2 * pr.used + 2 > pr.pool.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            pr.pool.push_back(a);
            pr.pool.push_back(b);
        }
        pair = pr.used++;
        if (pr.slot.size() < pr.used) pr.slot.resize(pr.used);
        pr.slot[pair] = slot_;
        cudaEventRecord(pr.pool[2 * pair], st);
    }
    ~ProfScope()
    {
        if (pair != (size_t)-1) cudaEventRecord(pr.pool[2 * pair + 1], st);
    }
};

// ----------------------------------------------------------------------------
// engines
// ----------------------------------------------------------------------------

struct sf_level_state {
    sf_grid grid;
    int N, S;
    float gamma[5];       // gamma[2] scaled for this level (reading R10)
    float4* s0[2];        // state, double buffered by frame parity
    float4* s1[2];
    float4* p0;           // prediction k+
    float4* p1;
    float4* t0;           // between propagation launches; then the solution
    float4* t1;           // between propagation launches; then Y-hat (as floats)
    void* block;          // one allocation holding the eight planes
};

struct EngineStream {
    int H, W, L;
    sf_params p;
    sf_level_state lv[SF_MAX_LEVELS];
    float* image;         // input/output slots (batches); null: the frame's pointers
    float* range;
    float* flow;
    float* inv;
    float* motion;        // Omega (rad/s) and a (m/s^2) over the next frame, device (6 floats)
};

struct Engine {
    std::vector<EngineStream> st;
    int flags = 0;
    int nf_max = kNfLimit;      // sub-iterations fused per propagation launch (tuned or set)
    sf_surrogate* surr = nullptr;   // when set, predicts every stream's top level instead of k_propagate
    int parity = 0;
    int initialised = 0;
    float dt_prev = 0.0f;
    int* status = nullptr;
    std::vector<Plan> prop;     // propagation launches
    Plan solve;                 // every level of every stream
    std::vector<Plan> smooth;   // cascade: depth d handles level L - 1 - d of every stream; parallel: one plan
    std::vector<Plan> recon;    // parallel: reconstruction of depth 1, 2, ... (coarse first)
    int update_mode = 1;        // 1: smoothing + reconstruction cascade; 2: all smoothing, then reconstruction
    int update_auto = 0;        // the tuner chooses update_mode
    int solve_t = kSolveT;      // tile edge of the solve launch
    int solve_auto = 0;         // the tuner chooses solve_t
    void* io = nullptr;         // slots of a batch
    float* motion = nullptr;    // every stream's motion slot (8 floats each), zeroed
    Profiler prof;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    float graph_dt[2] = {0.0f, 0.0f};
    int steps_plain = 0;
    // the surrogate's fallback (engine_surr_plans): one plain step of every
    // top level, the residual of the surrogate's prediction against it, and
    // the plain propagation gated per stream by residual > threshold
    float surr_thr_default = 1.0f;   // px/frame, for streams attached later
    void* surr_block = nullptr;
    bool surr_same_grid = false;     // every top level on one grid: one fused launch per 64 streams
    unsigned* surr_res = nullptr;    // per stream: the frame's residual (float bits), zeroed every frame
    float* surr_thr = nullptr;       // per stream: threshold (px/frame)
    unsigned* surr_cnt = nullptr;    // per stream: frames whose prediction fell back to the plain propagation
    Plan surr_one_plan;
    std::vector<Plan> surr_fb;       // gated plain propagation of the top levels (one per segment)

    int launches_per_step() const
    {
        int n = (int)prop.size() + 1;
        for (auto& p : smooth) n += p.nwork ? 1 : 0;
        for (auto& p : recon) n += p.nwork ? 1 : 0;
        if (surr) {   // per group of streams the fused network (features included); the check; the fallback segments
            const int groups = surr_same_grid ? ((int)st.size() + kNetMaxImg - 1) / kNetMaxImg : (int)st.size();
            n += groups + 1 + (int)surr_fb.size();
        }
        return n;
    }
};

namespace {

// the solve's tile edge: the parameter, else 16 when the levels' 32-pixel
// tiles fit in one wave (k_solve keeps 5 CTAs per SM resident), else 32; the
// autotuner times both when the parameter is 0
void engine_solve_tile(Engine& E, int param)
{
    if (param) {
        E.solve_t = param;
        return;
    }
    long tiles = 0;
    for (auto& s : E.st)
        for (int h = 0; h < s.L; ++h)
            tiles += (long)ceil_div(s.H >> h, kSolveT) * ceil_div(s.W >> h, kSolveT);
    E.solve_t = tiles <= 5L * kSmCount ? kSolveTSmall : kSolveT;
    E.solve_auto = (E.flags & SF_AUTOTUNE) != 0;
}

void engine_surr_free(Engine& E)
{
    free_plan(E.surr_one_plan);
    for (auto& pl : E.surr_fb) free_plan(pl);
    E.surr_fb.clear();
}

void engine_free(Engine& E)
{
    for (int q = 0; q < 2; ++q)
        if (E.graph[q]) cudaGraphExecDestroy(E.graph[q]);
    engine_surr_free(E);
    cudaFree(E.surr_block);
    for (auto& pl : E.prop) free_plan(pl);
    free_plan(E.solve);
    for (auto& pl : E.smooth) free_plan(pl);
    for (auto& pl : E.recon) free_plan(pl);
    for (auto& s : E.st)
        for (int h = 0; h < s.L; ++h) cudaFree(s.lv[h].block);
    cudaFree(E.io);
    cudaFree(E.motion);
    cudaFree(E.status);
}

int engine_levels(EngineStream& s, cudaStream_t st)
{
    for (int h = 0; h < s.L; ++h) {
        sf_level_state& lv = s.lv[h];
        const float sc = (float)(1 << h);
        lv.grid.H = s.H >> h;
        lv.grid.W = s.W >> h;
        lv.grid.fx = s.p.fx / sc; lv.grid.fy = s.p.fy / sc; lv.grid.cx = s.p.cx / sc; lv.grid.cy = s.p.cy / sc;
        lv.N = s.p.iters[h] > 0 ? s.p.iters[h] : std::max(1, (int)std::ceil(s.p.max_flow / sc));
        lv.S = s.p.smooth_iters[h];
        for (int k = 0; k < 5; ++k) lv.gamma[k] = s.p.gamma[k];
        const double dmu_c = (double)sc / (double)s.p.fx;   // reading R10
        lv.gamma[2] = (float)(s.p.gamma[2] * dmu_c * dmu_c);
        const size_t n = (size_t)lv.grid.H * lv.grid.W;
        lv.block = nullptr;
        if (cudaMalloc(&lv.block, 8 * n * sizeof(float4)) != cudaSuccess) { lv.block = nullptr; return SF_ENOMEM; }
        if (cudaMemsetAsync(lv.block, 0, 8 * n * sizeof(float4), st) != cudaSuccess) return SF_ECUDA;
        float4* b = (float4*)lv.block;
        lv.s0[0] = b; lv.s1[0] = b + n; lv.s0[1] = b + 2 * n; lv.s1[1] = b + 3 * n;
        lv.p0 = b + 4 * n; lv.p1 = b + 5 * n; lv.t0 = b + 6 * n; lv.t1 = b + 7 * n;
    }
    return SF_OK;
}

// The surrogate's fallback plans (nothing without a surrogate): every
// stream's top level once more with one plain sub-iteration (N = 1), in the
// propagation's residual mode (each tile reduces its largest difference to
// the surrogate's prediction into the stream's residual word instead of
// storing); and the plain propagation of the top levels
// in segments of at most nf_max sub-iterations (as the plain engine splits
// them), each job gated by its stream's residual word and threshold.  The
// state is already rescaled for a frame-time change when these run
// (engine_launches scales it in place for the surrogate), so no job rescales.
int engine_surr_plans(Engine& E, cudaStream_t st)
{
    engine_surr_free(E);
    if (!E.surr) return SF_OK;
    const int n = (int)E.st.size();
    if (!E.surr_block) {
        const size_t bytes = 3 * ((n * sizeof(unsigned) + 255) & ~(size_t)255);
        if (cudaMalloc(&E.surr_block, bytes) != cudaSuccess) { E.surr_block = nullptr; return SF_ENOMEM; }
        unsigned char* p = (unsigned char*)E.surr_block;
        const size_t wb = (n * sizeof(unsigned) + 255) & ~(size_t)255;
        E.surr_res = (unsigned*)p;
        E.surr_thr = (float*)(p + wb);
        E.surr_cnt = (unsigned*)(p + 2 * wb);
        std::vector<float> thr(n, E.surr_thr_default);
        if (cudaMemsetAsync(E.surr_res, 0, 3 * wb, st) != cudaSuccess) return SF_ECUDA;
        if (cudaMemcpyAsync(E.surr_thr, thr.data(), n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SF_ECUDA;
    }
    // one plain sub-iteration of every top level
    {
        std::vector<PropJob> jobs;
        std::vector<int4> work;
        size_t off = 0;
        for (auto& s : E.st) {
            sf_level_state& lv = s.lv[s.L - 1];
            PropJob j;
            std::memset(&j, 0, sizeof(j));
            j.g = make_grid(lv.grid);
            j.in0[0] = lv.s0[0]; j.in0[1] = lv.s0[1];
            j.resid_ref = lv.p0;                       // the surrogate's prediction
            j.resid_out = E.surr_res + (&s - E.st.data());
            j.nf = 1;
            j.dt = 1.0f;
            j.tiles_x = ceil_div(lv.grid.W, prop_tile(1));
            j.motion = s.motion;
            jobs.push_back(j);
            add_tiles(work, (int)jobs.size() - 1, lv.grid.H, lv.grid.W, prop_tile(1), prop_tile_h(1, prop_warps(1)));
            off += (size_t)lv.grid.H * lv.grid.W;
        }
        E.surr_one_plan.nf = 1;
        E.surr_one_plan.resid = true;
        E.surr_one_plan.warps = prop_warps(1);
        E.surr_one_plan.smem = prop_smem_bytes(E.surr_one_plan.warps);
        int r = upload_plan(jobs, work, E.surr_one_plan, st);
        if (r) return r;
    }
    // the gated plain propagation of the top levels
    int maxseg = 0;
    for (auto& s : E.st) maxseg = std::max(maxseg, ceil_div(s.lv[s.L - 1].N, E.nf_max));
    E.surr_fb.resize(maxseg);
    for (int k = 0; k < maxseg; ++k) {
        std::vector<PropJob> jobs;
        std::vector<int4> work;
        int nfl = 0;   // the launch's longest job sets its CTA shape
        for (auto& s : E.st) {
            const int N = s.lv[s.L - 1].N, nseg = ceil_div(N, E.nf_max);
            if (k < nseg) nfl = std::max(nfl, N / nseg + (k < N % nseg ? 1 : 0));
        }
        const int warps = prop_warps(nfl);
        for (int si = 0; si < n; ++si) {
            EngineStream& s = E.st[si];
            sf_level_state& lv = s.lv[s.L - 1];
            const int nseg = ceil_div(lv.N, E.nf_max);
            if (k >= nseg) continue;
            const int nf = lv.N / nseg + (k < lv.N % nseg ? 1 : 0);
            auto out_of = [&](int seg) { return ((nseg - 1 - seg) % 2) == 0 ? lv.p0 : lv.t0; };
            PropJob j;
            std::memset(&j, 0, sizeof(j));
            j.g = make_grid(lv.grid);
            if (k == 0) {
                j.in0[0] = lv.s0[0]; j.in0[1] = lv.s0[1];
            } else {
                j.in0[0] = j.in0[1] = out_of(k - 1);
            }
            j.out0 = out_of(k);
            j.nf = nf;
            j.dt = 1.0f / (float)lv.N;
            j.tiles_x = ceil_div(lv.grid.W, prop_tile(nf));
            j.motion = s.motion;
            j.gate = E.surr_res + si;
            j.gate_thr = E.surr_thr + si;
            j.gate_count = k == 0 ? E.surr_cnt + si : nullptr;
            jobs.push_back(j);
            add_tiles(work, (int)jobs.size() - 1, lv.grid.H, lv.grid.W, prop_tile(nf), prop_tile_h(nf, warps));
        }
        E.surr_fb[k].nf = nfl;
        E.surr_fb[k].warps = warps;
        E.surr_fb[k].smem = prop_smem_bytes(warps);
        int r = upload_plan(jobs, work, E.surr_fb[k], st);
        if (r) return r;
    }
    return SF_OK;
}

// The propagation job of segment k (of nseg) of level h of stream s: the
// last segment writes the prediction planes, earlier ones alternate with t0/t1
// (so segments k - 1 and k + 1 share a buffer), the first reads the state of
// the frame's parity and rescales w on load.
PropJob make_prop_job(const EngineStream& s, const sf_level_state& lv, bool top, int k, int nseg, int nf)
{
    auto out_of = [&](int seg, float4*& o0, float4*& o1) {
        const bool to_pred = ((nseg - 1 - seg) % 2) == 0;
        o0 = to_pred ? lv.p0 : lv.t0;
        o1 = to_pred ? lv.p1 : lv.t1;
    };
    PropJob j;
    std::memset(&j, 0, sizeof(j));
    j.g = make_grid(lv.grid);
    if (k == 0) {
        j.in0[0] = lv.s0[0]; j.in0[1] = lv.s0[1];
        j.in1[0] = top ? nullptr : lv.s1[0]; j.in1[1] = top ? nullptr : lv.s1[1];
        j.apply_wscale = 1;
    } else {
        float4 *o0, *o1;
        out_of(k - 1, o0, o1);
        j.in0[0] = j.in0[1] = o0;
        j.in1[0] = j.in1[1] = top ? nullptr : o1;
    }
    out_of(k, j.out0, j.out1);
    if (top) j.out1 = nullptr;
    j.nf = nf;
    j.dt = 1.0f / (float)lv.N;
    j.tiles_x = ceil_div(lv.grid.W, prop_tile(nf));
    j.motion = s.motion;
    return j;
}

// List schedule of the propagation of levels that need several segments.
// Launch k of the segment-per-launch schedule holds segment k of every level;
// a launch of more tiles than one wave leaves most SMs idle in its last wave
// (384 x 1248 at 8 sub-iterations per segment: 208 tiles, two waves on 148
// SMs, the second 40% full).  Here every (segment, tile) item goes into the
// first launch with room (one wave of CTAs) after all launches holding an item
// of the level's previous segment whose tile meets the item's region (values
// it reads) or whose region meets the item's tile (values it overwrites:
// segments k - 1 and k + 1 write the same buffer).  So within a launch no
// item reads what another one writes, and items of later segments start while
// the remaining tiles of earlier segments still run.  Used when its one-wave
// launches come out ahead of the segment-per-launch schedule's waves, counting
// a tenth of a wave per launch; returns false otherwise.
bool engine_prop_list_schedule(Engine& E, cudaStream_t st, int& rc)
{
    const int nfmax = E.nf_max;
    struct Seg { int s, h, k, nseg, nf, job, t0; };   // t0: first item of the segment
    std::vector<Seg> segs;
    std::vector<PropJob> jobs;
    int nf_long = 0;
    for (size_t si = 0; si < E.st.size(); ++si) {
        const EngineStream& s = E.st[si];
        for (int h = 0; h < s.L; ++h) {
            if (h == s.L - 1 && E.surr) continue;
            const int N = s.lv[h].N, nseg = ceil_div(N, nfmax);
            for (int k = 0; k < nseg; ++k) {
                const int nf = N / nseg + (k < N % nseg ? 1 : 0);
                nf_long = std::max(nf_long, nf);
                segs.push_back({(int)si, h, k, nseg, nf, (int)jobs.size(), 0});
                jobs.push_back(make_prop_job(s, s.lv[h], h == s.L - 1, k, nseg, nf));
            }
        }
    }
    const int warps = prop_warps(nf_long);
    const int cap = kSmCount * (warps == kPrWarpsMax ? 1 : 2);   // CTAs of one wave
    // the waves of the segment-per-launch schedule (launch k's CTA shape set by
    // its own longest job)
    int waves_plain = 0, maxk = 0;
    for (const Seg& g : segs) maxk = std::max(maxk, g.k);
    if (maxk == 0) return false;
    for (int k = 0; k <= maxk; ++k) {
        int nfk = 0;
        for (const Seg& g : segs)
            if (g.k == k) nfk = std::max(nfk, g.nf);
        const int wk = prop_warps(nfk);
        long n = 0;
        for (const Seg& g : segs)
            if (g.k == k) {
                const sf_level_state& lv = E.st[g.s].lv[g.h];
                n += (long)ceil_div(lv.grid.H, prop_tile_h(g.nf, wk)) * ceil_div(lv.grid.W, prop_tile(g.nf));
            }
        const long capk = (long)kSmCount * (wk == kPrWarpsMax ? 1 : 2);
        waves_plain += (int)((n + capk - 1) / capk);
    }
    // items in order of segment, then level and raster order; launch of each
    std::vector<int4> item;        // (job, y0, x0, launch)
    std::vector<int> load;
    for (int k = 0; k <= maxk; ++k) {
        for (size_t gi = 0; gi < segs.size(); ++gi) {
            Seg& g = segs[gi];
            if (g.k != k) continue;
            const sf_level_state& lv = E.st[g.s].lv[g.h];
            const int TW = prop_tile(g.nf), TH = prop_tile_h(g.nf, warps);
            const Seg* pv = k ? &segs[gi - 1] : nullptr;   // the level's previous segment
            const int PW = pv ? prop_tile(pv->nf) : 1, PH = pv ? prop_tile_h(pv->nf, warps) : 1;
            const int ptx = pv ? ceil_div(lv.grid.W, PW) : 0, pty = pv ? ceil_div(lv.grid.H, PH) : 0;
            g.t0 = (int)item.size();
            for (int y0 = 0; y0 < lv.grid.H; y0 += TH)
                for (int x0 = 0; x0 < lv.grid.W; x0 += TW) {
                    int earliest = 0;
                    if (pv) {
                        const int m = std::max(g.nf, pv->nf);   // the item's tile grown by the larger halo
                        const int ya = std::max(0, y0 - m), yb = std::min(lv.grid.H, y0 + TH + m) - 1;
                        const int xa = std::max(0, x0 - m), xb = std::min(lv.grid.W, x0 + TW + m) - 1;
                        for (int py = ya / PH; py <= std::min(pty - 1, yb / PH); ++py)
                            for (int px = xa / PW; px <= std::min(ptx - 1, xb / PW); ++px)
                                earliest = std::max(earliest, item[pv->t0 + py * ptx + px].w + 1);
                    }
                    int L = earliest;
                    while (L < (int)load.size() && load[L] >= cap) ++L;
                    if (L >= (int)load.size()) load.resize(L + 1, 0);
                    ++load[L];
                    item.push_back(make_int4(g.job, y0, x0, L));
                }
        }
    }
    // a launch costs about a tenth of a wave beyond its CTAs' work (its start and
    // the drain of its last wave): keep the list schedule only where its waves
    // and the extra launches together still come out ahead
    if (11 * (int)load.size() >= 10 * waves_plain + (maxk + 1)) return false;
    // one plan per launch: the launch's jobs (renumbered), longest tiles first
    const int nl = (int)load.size();
    E.prop.resize(nl);
    for (int L = 0; L < nl && !rc; ++L) {
        std::vector<PropJob> lj;
        std::vector<int> map(jobs.size(), -1);
        std::vector<int4> work;
        bool c8 = false;
        int nfl = 0;
        for (int want = nfmax; want >= 1; --want)
            for (const int4& it : item) {
                if (it.w != L || jobs[it.x].nf != want) continue;
                if (map[it.x] < 0) {
                    map[it.x] = (int)lj.size();
                    lj.push_back(jobs[it.x]);
                    c8 |= jobs[it.x].out1 != nullptr;
                    nfl = std::max(nfl, want);
                }
                work.push_back(make_int4(map[it.x], it.y, it.z, 0));
            }
        E.prop[L].c8 = c8;
        E.prop[L].nf = nfl;
        E.prop[L].warps = warps;
        E.prop[L].smem = prop_smem_bytes(warps);
        rc = upload_plan(lj, work, E.prop[L], st);
    }
    return true;
}

int engine_prop_plans(Engine& E, cudaStream_t st)
{
    for (auto& pl : E.prop) free_plan(pl);
    E.prop.clear();
    const int nfmax = E.nf_max;
    {
        int rc = SF_OK;
        if (engine_prop_list_schedule(E, st, rc)) return rc ? rc : engine_surr_plans(E, st);
    }
    // ---- propagation: level h of stream s runs ceil(N / nfmax) launches;
    // launch k holds segment k of every (stream, level) that has one.
    int maxseg = 0;
    for (auto& s : E.st)
        for (int h = 0; h < s.L - (E.surr ? 1 : 0); ++h) maxseg = std::max(maxseg, ceil_div(s.lv[h].N, nfmax));
    E.prop.resize(maxseg);
    for (int k = 0; k < maxseg; ++k) {
        std::vector<PropJob> jobs;
        std::vector<int4> work;
        bool c8 = false;
        int nfl = 0;   // the longest job's sub-iterations: it sets the launch's CTA shape
        for (auto& s : E.st)
            for (int h = 0; h < s.L; ++h) {
                const int N = s.lv[h].N, nseg = ceil_div(N, nfmax);
                if (k < nseg && !(h == s.L - 1 && E.surr)) nfl = std::max(nfl, N / nseg + (k < N % nseg ? 1 : 0));
            }
        const int warps = prop_warps(nfl);
        for (int want = nfmax; want >= 1; --want) {   // longest tiles (most passes) first
            for (auto& s : E.st) {
                for (int h = 0; h < s.L; ++h) {
                    sf_level_state& lv = s.lv[h];
                    const int nseg = ceil_div(lv.N, nfmax);
                    if (k >= nseg) continue;
                    const int nf = lv.N / nseg + (k < lv.N % nseg ? 1 : 0);
                    if (nf != want) continue;
                    const bool top = h == s.L - 1;
                    if (top && E.surr) continue;
                    jobs.push_back(make_prop_job(s, lv, top, k, nseg, nf));
                    add_tiles(work, (int)jobs.size() - 1, lv.grid.H, lv.grid.W, prop_tile(nf), prop_tile_h(nf, warps));
                    c8 |= !top;
                }
            }
        }
        E.prop[k].c8 = c8;
        E.prop[k].nf = nfl;
        E.prop[k].warps = warps;
        E.prop[k].smem = prop_smem_bytes(warps);
        int r = upload_plan(jobs, work, E.prop[k], st);
        if (r) return r;
    }
    return engine_surr_plans(E, st);
}

int engine_smooth_plans(Engine& E, cudaStream_t st);

int engine_update_plans(Engine& E, cudaStream_t st)
{
    // ---- solve: every level of every stream, one solve_t x solve_t tile per CTA
    {
        free_plan(E.solve);
        std::vector<SolveJob> jobs;
        std::vector<int4> work;
        for (auto& s : E.st) {
            for (int h = s.L - 1; h >= 0; --h) {
                sf_level_state& lv = s.lv[h];
                SolveJob j;
                std::memset(&j, 0, sizeof(j));
                j.g = make_grid(lv.grid);
                j.level = h + 1;
                j.top = h == s.L - 1;
                j.g1 = lv.gamma[0]; j.g2 = lv.gamma[1]; j.g3 = lv.gamma[2]; j.g4 = lv.gamma[3]; j.g5 = lv.gamma[4];
                j.inv45 = 1.0f / (j.g4 + j.g5);
                j.inv5 = 1.0f / j.g5;
                for (int q = 0; q < 2; ++q) { j.s0_cur[q] = lv.s0[q]; j.s1_cur[q] = lv.s1[q]; }
                j.p0 = lv.p0;
                j.p1 = lv.p1;
                j.x_out = lv.t0;
                j.y_out = (float*)lv.t1;
                j.image = s.image;
                j.range = s.range;
                j.H1 = s.H;
                j.W1 = s.W;
                j.lambda_ref = s.p.lambda_ref;
                j.tiles_x = ceil_div(lv.grid.W, E.solve_t);
                jobs.push_back(j);
                add_tiles(work, (int)jobs.size() - 1, lv.grid.H, lv.grid.W, E.solve_t, E.solve_t);
            }
        }
        int r = upload_plan(jobs, work, E.solve, st);
        if (r) return r;
        E.solve.tile = E.solve_t;
    }
    return engine_smooth_plans(E, st);
}

// smoothing (+ reconstruction) plans of the engine's update mode
int engine_smooth_plans(Engine& E, cudaStream_t st)
{
    for (auto& pl : E.smooth) free_plan(pl);
    for (auto& pl : E.recon) free_plan(pl);
    E.smooth.clear();
    E.recon.clear();
    int maxL = 0;
    for (auto& s : E.st) maxL = std::max(maxL, s.L);
    const bool parallel = E.update_mode == 2;
    // cascade: depth d in plan d; parallel: every depth in plan 0, lower levels deferred
    E.smooth.resize(parallel ? 1 : maxL);
    for (int d = 0; d < maxL; ++d) {
        const int plan = parallel ? 0 : d;
        if (parallel && d > 0) continue;   // plan 0 takes every depth below
        std::vector<SmoothJob> jobs;
        std::vector<int4> work;
        size_t smem = 0;
        for (int dd = d; dd < (parallel ? maxL : d + 1); ++dd)
        for (auto& s : E.st) {
            const int h = s.L - 1 - dd;
            if (h < 0) continue;
            sf_level_state& lv = s.lv[h];
            SmoothJob j;
            std::memset(&j, 0, sizeof(j));
            j.H = lv.grid.H;
            j.W = lv.grid.W;
            j.S = lv.S;
            j.top = h == s.L - 1;
            j.x_in = lv.t0;
            j.y_in = (const float*)lv.t1;
            for (int q = 0; q < 2; ++q) {
                j.s0_new[q] = lv.s0[q];
                j.s1_new[q] = lv.s1[q];
                j.s0c[q] = j.top ? nullptr : s.lv[h + 1].s0[q];
            }
            if (!j.top) { j.Hc = s.lv[h + 1].grid.H; j.Wc = s.lv[h + 1].grid.W; }
            if (h == 0) {
                j.flow_out = s.flow;
                j.invdepth_out = s.inv;
                j.frame_outputs = s.image == nullptr;   // single-stream filter: per-frame output pointers
            }
            if (parallel && !j.top) {
                j.defer = 1;
                j.s0c[0] = j.s0c[1] = nullptr;
                j.flow_out = j.invdepth_out = nullptr;
                j.frame_outputs = 0;
            }
            j.tiles_x = ceil_div(lv.grid.W, kSmoothT);
            jobs.push_back(j);
            add_tiles(work, (int)jobs.size() - 1, lv.grid.H, lv.grid.W, kSmoothT, kSmoothT);
            smem = std::max(smem, smooth_smem_bytes(j.S));
        }
        E.smooth[plan].smem = smem;
        int r = upload_plan(jobs, work, E.smooth[plan], st);
        if (r) return r;
    }
    if (!parallel) return SF_OK;
    // reconstruction of the deferred levels, depth 1 (just below the top) first
    E.recon.resize(std::max(0, maxL - 1));
    for (int d = 1; d < maxL; ++d) {
        std::vector<ReconJob> jobs;
        std::vector<int4> work;
        for (auto& s : E.st) {
            const int h = s.L - 1 - d;
            if (h < 0) continue;
            sf_level_state& lv = s.lv[h];
            ReconJob j;
            std::memset(&j, 0, sizeof(j));
            j.H = lv.grid.H; j.W = lv.grid.W;
            j.Hc = s.lv[h + 1].grid.H; j.Wc = s.lv[h + 1].grid.W;
            for (int q = 0; q < 2; ++q) { j.s0[q] = lv.s0[q]; j.s0c[q] = s.lv[h + 1].s0[q]; }
            if (h == 0) {
                j.flow_out = s.flow;
                j.invdepth_out = s.inv;
                j.frame_outputs = s.image == nullptr;
            }
            jobs.push_back(j);
            const int n = lv.grid.H * lv.grid.W;
            for (int p0 = 0; p0 < n; p0 += kReconChunk) work.push_back(make_int4((int)jobs.size() - 1, p0, 0, 0));
        }
        int r = upload_plan(jobs, work, E.recon[d - 1], st);
        if (r) return r;
    }
    return SF_OK;
}

// The autotuner: time one frame's propagation launches for every nf_max in
// {8, 6, 4, 3, 2} that splits the levels' N_h into a different set of launches
// (12 frames after 2 warm-up frames, CUDA events on the engine's stream; two
// interleaved rounds, each candidate keeping its faster) and keep the fastest.  It runs on the engine's zero state: the kernel has no
// data-dependent branches, so the timing is that of any state, and the
// propagation of zeros writes zeros, so the engine is left as created.
int engine_update_launches(Engine& E, const UpdArgs& a, float dt, float* flow, float* inv, int slot, cudaStream_t st);
int net_forward(sf_surrogate* s, const Grid& g, int n, const float4* const* s0, float4* const* p0, cudaStream_t st);

constexpr int kTuneRounds = 2;

int engine_tune(Engine& E, cudaStream_t st)
{
    const int cand[] = {8, 6, 4, 3, 2};
    std::vector<std::vector<int>> seen;
    int best = E.nf_max, r = SF_OK;
    float best_ms = -1.0f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = SF_ECUDA;
    const int flags = E.flags & ~(SF_CHECK_CFL | SF_CHECK_FINITE);
    // every candidate is timed in kTuneRounds interleaved rounds and keeps its
    // fastest, so that one disturbed measurement cannot decide the choice
    std::vector<int> nfs;
    for (int nf : cand) {
        std::vector<int> sig;
        for (auto& s : E.st)
            for (int h = 0; h < s.L; ++h) sig.push_back(ceil_div(s.lv[h].N, nf));
        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
        seen.push_back(sig);
        nfs.push_back(nf);
    }
    std::vector<float> nf_ms(nfs.size(), -1.0f);
    for (int round = 0; round < kTuneRounds && nfs.size() > 1; ++round) {
        for (size_t c = 0; c < nfs.size() && !r; ++c) {
            E.nf_max = nfs[c];
            r = engine_prop_plans(E, st);
            for (int it = 0; it < 14 && !r; ++it) {
                if (it == 2 && cudaEventRecord(e0, st) != cudaSuccess) r = SF_ECUDA;
                for (auto& pl : E.prop)
                    if (!r) r = launch_propagate(pl, 0, 1.0f, flags, nullptr, st);
            }
            if (!r && cudaEventRecord(e1, st) != cudaSuccess) r = SF_ECUDA;
            if (!r && cudaEventSynchronize(e1) != cudaSuccess) r = SF_ECUDA;
            float ms = 0.0f;
            if (!r && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = SF_ECUDA;
            if (!r && (nf_ms[c] < 0.0f || ms < nf_ms[c])) nf_ms[c] = ms;
        }
    }
    for (size_t c = 0; c < nfs.size(); ++c)
        if (best_ms < 0.0f || (nf_ms[c] >= 0.0f && nf_ms[c] < best_ms)) { best_ms = nf_ms[c]; best = nfs[c]; }
    if (r) { if (e0) cudaEventDestroy(e0); if (e1) cudaEventDestroy(e1); return r; }
    E.nf_max = best;
    r = engine_prop_plans(E, st);
    // the update's form and the solve's tile edge, where the parameters leave
    // them open: time whole frames (the propagation launches just chosen, then
    // solve + smoothing (+ reconstruction)) for every combination on the zero
    // state (zero inputs and outputs kept in scratch buffers; the state stays
    // zero) and keep the fastest.  Whole frames, because a solve launch of
    // about one wave overlaps the propagation launch before it.
    int maxL = 0;
    size_t npx = 0;
    for (auto& es : E.st) { maxL = std::max(maxL, es.L); npx = std::max(npx, (size_t)es.H * es.W); }
    std::vector<int> modes, tiles;
    if (E.update_auto && maxL >= 2) modes = {1, 2};
    else modes = {E.update_mode};
    if (E.solve_auto) tiles = {kSolveT, kSolveTSmall};
    else tiles = {E.solve_t};
    if (!r && modes.size() * tiles.size() > 1) {
        float* scratch = nullptr;
        if (cudaMalloc(&scratch, 6 * npx * sizeof(float)) != cudaSuccess) scratch = nullptr, r = SF_ENOMEM;
        if (!r) r = cudaMemsetAsync(scratch, 0, 6 * npx * sizeof(float), st) == cudaSuccess ? SF_OK : SF_ECUDA;
        UpdArgs a;
        std::memset(&a, 0, sizeof(a));
        a.image = scratch;
        a.range = scratch + npx;
        a.H1 = E.st[0].H;
        a.W1 = E.st[0].W;
        a.lambda_ref = E.st[0].p.lambda_ref;
        std::vector<std::pair<int, int>> combos;
        for (int mode : modes)
            for (int tile : tiles) combos.emplace_back(mode, tile);
        std::vector<float> combo_ms(combos.size(), -1.0f);
        for (int round = 0; round < kTuneRounds; ++round) {
            for (size_t c = 0; c < combos.size() && !r; ++c) {
                E.update_mode = combos[c].first;
                E.solve_t = combos[c].second;
                r = engine_update_plans(E, st);
                for (int it = 0; it < 14 && !r; ++it) {
                    if (it == 2 && cudaEventRecord(e0, st) != cudaSuccess) r = SF_ECUDA;
                    for (auto& pl : E.prop)
                        if (!r) r = launch_propagate(pl, 0, 1.0f, flags, nullptr, st);
                    a.parity = it & 1;
                    if (!r) r = engine_update_launches(E, a, 1.0f, scratch + 2 * npx, scratch + 5 * npx, 0, st);
                }
                if (!r && cudaEventRecord(e1, st) != cudaSuccess) r = SF_ECUDA;
                if (!r && cudaEventSynchronize(e1) != cudaSuccess) r = SF_ECUDA;
                float ms = 0.0f;
                if (!r && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = SF_ECUDA;
                if (!r && (combo_ms[c] < 0.0f || ms < combo_ms[c])) combo_ms[c] = ms;
            }
        }
        float best_u = -1.0f;
        int best_mode = modes[0], best_tile = tiles[0];
        for (size_t c = 0; c < combos.size(); ++c)
            if (combo_ms[c] >= 0.0f && (best_u < 0.0f || combo_ms[c] < best_u)) {
                best_u = combo_ms[c];
                best_mode = combos[c].first;
                best_tile = combos[c].second;
            }
        if (!r && cudaStreamSynchronize(st) != cudaSuccess) r = SF_ECUDA;
        cudaFree(scratch);
        if (!r) {
            E.update_mode = best_mode;
            E.solve_t = best_tile;
            r = engine_update_plans(E, st);
        }
        if (!r && cudaMemsetAsync(E.status, 0, sizeof(int), st) != cudaSuccess) r = SF_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return r;
}

// create the streams' levels, the status word and the plans
int engine_init(Engine& E)
{
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SF_ECUDA;
    int r = SF_OK;
    for (auto& s : E.st) {
        r = engine_levels(s, st);
        if (r) break;
    }
    if (!r && cudaMalloc(&E.motion, E.st.size() * 8 * sizeof(float)) != cudaSuccess) { E.motion = nullptr; r = SF_ENOMEM; }
    if (!r) r = cudaMemsetAsync(E.motion, 0, E.st.size() * 8 * sizeof(float), st) == cudaSuccess ? SF_OK : SF_ECUDA;
    for (size_t k = 0; k < E.st.size() && !r; ++k) E.st[k].motion = E.motion + 8 * k;
    if (!r && cudaMalloc(&E.status, sizeof(int)) != cudaSuccess) { E.status = nullptr; r = SF_ENOMEM; }
    if (!r) r = cudaMemsetAsync(E.status, 0, sizeof(int), st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) r = engine_prop_plans(E, st);
    if (!r) r = engine_update_plans(E, st);
    if (!r && (E.flags & SF_AUTOTUNE)) r = engine_tune(E, st);
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
    cudaStreamDestroy(st);
    return r;
}

// the update of one frame: solve, smoothing (+ reconstruction) launches
int engine_update_launches(Engine& E, const UpdArgs& a, float dt, float* flow, float* inv, int slot, cudaStream_t st)
{
    int r;
    {
        NvtxRange nv("sf update: models + 3x3 solve + blend, every level");
        ProfScope ps(E.prof, slot++, st);
        r = launch_solve(E.solve, a, st);
        if (r) return r;
    }
    const int check = (E.flags & SF_CHECK_FINITE) != 0;
    static const char* const kSmoothNames[] = {"sf smoothing + reconstruction: top level",
                                               "sf smoothing + reconstruction: top level - 1",
                                               "sf smoothing + reconstruction: top level - 2",
                                               "sf smoothing + reconstruction: top level - 3"};
    int depth = 0;
    for (auto& pl : E.smooth) {
        if (!pl.nwork) continue;
        NvtxRange nv(E.update_mode == 2 ? "sf smoothing: every level" : kSmoothNames[std::min(depth, 3)]);
        ++depth;
        ProfScope ps(E.prof, slot++, st);
        r = launch_smooth(pl, a.parity ^ 1, 1.0f / dt, check, E.status, flow, inv, st);
        if (r) return r;
    }
    for (auto& pl : E.recon) {
        if (!pl.nwork) continue;
        NvtxRange nv("sf reconstruction of one level");
        ProfScope ps(E.prof, slot++, st);
        r = launch_recon(pl, a.parity ^ 1, 1.0f / dt, check, E.status, flow, inv, st);
        if (r) return r;
    }
    return SF_OK;
}

// the launches of one frame (no host synchronisation; capturable)
// inputs: an event the update waits for (inputs still being copied in while
// the propagation, which reads only the state, runs), or null
int engine_launches(Engine& E, const float* image, const float* range, float dt, float wscale, float* flow,
                    float* inv, cudaStream_t st, cudaEvent_t inputs = nullptr)
{
    UpdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = image;
    a.range = range;
    a.H1 = E.st[0].H;
    a.W1 = E.st[0].W;
    a.lambda_ref = E.st[0].p.lambda_ref;
    a.parity = E.parity;
    a.init = !E.initialised;
    NvtxRange frame("sf frame");
    int slot = 0, r;
    if (!a.init) {
        for (auto& pl : E.prop) {
            NvtxRange nv("sf prediction: propagation launch (every level of every stream)");
            ProfScope ps(E.prof, slot++, st);
            r = launch_propagate(pl, E.parity, wscale, E.flags, E.status, st, dt);
            if (r) return r;
        }
        if (E.surr) {
            NvtxRange nv("sf prediction: surrogate network (top levels)");
            ProfScope ps(E.prof, slot++, st);
            for (auto& s : E.st) {
                sf_level_state& lv = s.lv[s.L - 1];
                const size_t n = (size_t)lv.grid.H * lv.grid.W;
                if (wscale != 1.0f) {
                    k_scale_w<<<(int)std::min<size_t>((n + 255) / 256, kSmCount * 8), 256, 0, st>>>(lv.s0[E.parity], n,
                                                                                              wscale);
                    if (last_error()) return SF_ECUDA;
                }
            }
            // one fused launch per group of up to kNetMaxImg streams on one grid
            // (else one per stream), into the engine's own features buffer
            const int ns = (int)E.st.size();
            const int group = E.surr_same_grid ? kNetMaxImg : 1;
            for (int k0 = 0; k0 < ns && !r; k0 += group) {
                const int m = std::min(group, ns - k0);
                const float4* in[kNetMaxImg];
                float4* out[kNetMaxImg];
                for (int k = 0; k < m; ++k) {
                    sf_level_state& lv = E.st[k0 + k].lv[E.st[k0 + k].L - 1];
                    in[k] = lv.s0[E.parity];
                    out[k] = lv.p0;
                }
                sf_level_state& lv0 = E.st[k0].lv[E.st[k0].L - 1];
                r = net_forward(E.surr, make_grid(lv0.grid), m, in, out, st);
            }
            if (r) return r;
        }
        if (E.surr) {
            // the fallback: residual against one plain step, then the plain
            // propagation of every stream whose residual exceeds its threshold
            // (CTAs of the other streams return at once); no host decision
            NvtxRange nv("sf prediction: surrogate check and gated plain fallback");
            ProfScope ps(E.prof, slot++, st);
            if (cudaMemsetAsync(E.surr_res, 0, E.st.size() * sizeof(unsigned), st) != cudaSuccess) return SF_ECUDA;
            // one plain sub-iteration of every top level, reduced on the fly to each
            // stream's largest difference to the surrogate's prediction
            r = launch_propagate(E.surr_one_plan, E.parity, 1.0f, E.flags & ~SF_CHECK_CFL, nullptr, st, dt);
            if (r) return r;
            for (auto& pl : E.surr_fb) {
                r = launch_propagate(pl, E.parity, 1.0f, E.flags, E.status, st, dt);
                if (r) return r;
            }
        }
    } else {
        slot = (int)E.prop.size() + (E.surr ? 2 : 0);
    }
    if (inputs && cudaStreamWaitEvent(st, inputs, 0) != cudaSuccess) return SF_ECUDA;
    return engine_update_launches(E, a, dt, flow, inv, slot, st);
}

int engine_status(Engine& E)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return SF_ECUDA;
    int s = 0;
    if (cudaMemcpy(&s, E.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SF_ECUDA;
    if (cudaMemset(E.status, 0, sizeof(int)) != cudaSuccess) return SF_ECUDA;
    if (s & kStatusTimeout) return SF_ETIMEOUT;
    if (s & kStatusNonFinite) return SF_ENONFINITE;
    if (s & kStatusCfl) return SF_WARN_CFL;
    return SF_OK;
}

}  // namespace

// staging slots of the pipelined host-buffer steps: frame k uses slot k % kRing;
// frame k's completion is marked by event k % kDone (host waits)
constexpr int kRing = 3;
constexpr int kDone = 64;

struct sf_ctx {
    Engine E;
    // staging for sf_step_host
    float* stage_image = nullptr;
    float* stage_range = nullptr;
    float* stage_flow = nullptr;
    float* stage_inv = nullptr;
    cudaStream_t stage_copy = nullptr;                      // input copies, beside the propagation
    cudaEvent_t stage_free = nullptr, stage_in = nullptr;   // staging free / inputs copied
    // sf_submit_host: per slot image, range, flow (3 planes), inverse depth on
    // the device; input copies on pipe_in, output copies on pipe_out, the step
    // on the caller's stream; events order the three and guard slot reuse
    float* ring[kRing] = {};
    cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
    cudaEvent_t ev_in[kRing] = {}, ev_run[kRing] = {}, ev_out[kRing] = {};
    cudaEvent_t ev_done[kDone] = {};
    long long submitted = 0;
};

struct sf_batch {
    Engine E;
};

namespace {

void destroy_ctx(sf_ctx* c)
{
    if (!c) return;
    if (c->pipe_in) cudaStreamSynchronize(c->pipe_in);
    if (c->pipe_out) cudaStreamSynchronize(c->pipe_out);
    engine_free(c->E);
    cudaFree(c->stage_image);
    cudaFree(c->stage_range);
    cudaFree(c->stage_flow);
    cudaFree(c->stage_inv);
    if (c->stage_copy) {
        cudaStreamSynchronize(c->stage_copy);
        cudaStreamDestroy(c->stage_copy);
    }
    if (c->stage_free) cudaEventDestroy(c->stage_free);
    if (c->stage_in) cudaEventDestroy(c->stage_in);
    for (int k = 0; k < kRing; ++k) {
        cudaFree(c->ring[k]);
        if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
        if (c->ev_run[k]) cudaEventDestroy(c->ev_run[k]);
        if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
    }
    for (int k = 0; k < kDone; ++k)
        if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
    if (c->pipe_in) cudaStreamDestroy(c->pipe_in);
    if (c->pipe_out) cudaStreamDestroy(c->pipe_out);
    delete c;
}

// first sf_submit_host: the staging ring, the two copy streams (non-blocking,
// so that they never wait on the legacy default stream implicitly) and the
// events (no timing)
int pipe_init(sf_ctx* c)
{
    const size_t n = (size_t)c->E.st[0].H * c->E.st[0].W;
    for (int k = 0; k < kRing; ++k) {
        if (cudaMalloc(&c->ring[k], 6 * n * sizeof(float)) != cudaSuccess) return SF_ENOMEM;
        if (cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_run[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming) != cudaSuccess)
            return SF_ECUDA;
    }
    for (int k = 0; k < kDone; ++k)
        if (cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming) != cudaSuccess) return SF_ECUDA;
    if (cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking) != cudaSuccess)
        return SF_ECUDA;
    return SF_OK;
}

void destroy_batch(sf_batch* b)
{
    if (!b) return;
    engine_free(b->E);
    delete b;
}

}  // namespace

// ----------------------------------------------------------------------------
// C ABI: single-stream filter
// ----------------------------------------------------------------------------

extern "C" {

int sf_params_default(sf_params* p, int H, int W, int levels)
{
    if (!p || H <= 0 || W <= 0 || levels < 1 || levels > SF_MAX_LEVELS) return SF_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->fx = p->fy = 0.5f * (float)W;
    p->cx = 0.5f * (float)W;
    p->cy = 0.5f * (float)H;
    p->max_flow = 1.0f;
    for (int h = 0; h < SF_MAX_LEVELS; ++h) {
        p->iters[h] = 0;
        p->smooth_iters[h] = h == 0 ? 2 : 4;
    }
    p->gamma[0] = 1.0f;
    p->gamma[1] = 1.0f;
    p->gamma[2] = 1e-2f;
    p->gamma[3] = 1.0f;
    p->gamma[4] = 1.0f;
    p->lambda_ref = 1.0f;
    p->flags = SF_CHECK_CFL;
    return SF_OK;
}

int sf_create(int H, int W, int levels, const sf_params* p, sf_ctx** out)
{
    if (out) *out = nullptr;
    if (!out) return SF_EINVAL;
    int r = check_params(H, W, levels, p);
    if (r) return r;
    sf_ctx* c = new (std::nothrow) sf_ctx();
    if (!c) return SF_ENOMEM;
    c->E.st.resize(1);
    EngineStream& s = c->E.st[0];
    std::memset(&s, 0, sizeof(s));
    s.H = H; s.W = W; s.L = levels; s.p = *p;
    c->E.flags = p->flags;
    c->E.nf_max = p->nf_max ? p->nf_max : kNfLimit;
    c->E.update_mode = p->update_mode ? p->update_mode : 1;
    c->E.update_auto = p->update_mode == 0 && (p->flags & SF_AUTOTUNE);
    engine_solve_tile(c->E, p->solve_tile);
    r = engine_init(c->E);
    if (r) { destroy_ctx(c); return r; }
    *out = c;
    return SF_OK;
}

int sf_reset(sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    c->E.initialised = 0;
    return SF_OK;
}

namespace {

int step_impl(sf_ctx* c, const float* image, const float* range, float dt, float* flow_out, float* invdepth_out,
              cudaStream_t st, cudaEvent_t inputs)
{
    if (!c || !image || !range || !(dt > 0.0f) || !std::isfinite(dt)) return SF_EINVAL;
    Engine& E = c->E;
    const float wscale = E.initialised ? dt / E.dt_prev : 1.0f;   // reading R9
    const int r = engine_launches(E, image, range, dt, wscale, flow_out, invdepth_out, st, inputs);
    if (r) return r;
    E.parity ^= 1;
    E.initialised = 1;
    E.dt_prev = dt;
    return SF_OK;
}

}  // namespace

int sf_step(sf_ctx* c, const float* image, const float* range, float dt, float* flow_out, float* invdepth_out,
            void* stream)
{
    return step_impl(c, image, range, dt, flow_out, invdepth_out, (cudaStream_t)stream, nullptr);
}

int sf_step_host(sf_ctx* c, const float* image, const float* range, float dt, float* flow_out, float* invdepth_out,
                 void* stream)
{
    if (!c || !image || !range || !(dt > 0.0f) || !std::isfinite(dt)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->E.st[0].H * c->E.st[0].W;
    if (!c->stage_image) {
        if (cudaMalloc(&c->stage_image, n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&c->stage_range, n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&c->stage_flow, 3 * n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&c->stage_inv, n * sizeof(float)) != cudaSuccess)
            return SF_ENOMEM;
    }
    if (!c->stage_copy) {
        if (cudaStreamCreateWithFlags(&c->stage_copy, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->stage_in, cudaEventDisableTiming) != cudaSuccess)
            return SF_ECUDA;
    }
    // the inputs go in on a side stream once the staging is free (earlier work
    // on the caller's stream done with it), beside the propagation, which reads
    // only the state; the update waits for them
    if (cudaEventRecord(c->stage_free, st) != cudaSuccess ||
        cudaStreamWaitEvent(c->stage_copy, c->stage_free, 0) != cudaSuccess ||
        cudaMemcpyAsync(c->stage_image, image, n * sizeof(float), cudaMemcpyHostToDevice, c->stage_copy) != cudaSuccess ||
        cudaMemcpyAsync(c->stage_range, range, n * sizeof(float), cudaMemcpyHostToDevice, c->stage_copy) != cudaSuccess ||
        cudaEventRecord(c->stage_in, c->stage_copy) != cudaSuccess) {
        cudaStreamSynchronize(c->stage_copy);   // no copy from the caller's buffers outlives the call
        return SF_ECUDA;
    }
    int r = step_impl(c, c->stage_image, c->stage_range, dt, flow_out ? c->stage_flow : nullptr,
                      invdepth_out ? c->stage_inv : nullptr, st, c->stage_in);
    if (r) {
        cudaStreamSynchronize(c->stage_copy);
        return r;
    }
    if (flow_out && cudaMemcpyAsync(flow_out, c->stage_flow, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess)
        return SF_ECUDA;
    if (invdepth_out &&
        cudaMemcpyAsync(invdepth_out, c->stage_inv, n * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SF_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
}

int sf_submit_host(sf_ctx* c, const float* image, const float* range, float dt, float* flow_out,
                   float* invdepth_out, void* stream, long long* ticket)
{
    if (ticket) *ticket = -1;
    if (!c || !image || !range || !(dt > 0.0f) || !std::isfinite(dt)) return SF_EINVAL;
    if (!c->pipe_in) {
        const int r = pipe_init(c);
        if (r) return r;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->E.st[0].H * c->E.st[0].W;
    const long long k = c->submitted;
    const int s = (int)(k % kRing);
    float* img = c->ring[s];
    float* rng = img + n;
    float* flow = rng + n;
    float* inv = flow + 3 * n;
    // inputs: the slot was last read by the step of frame k - kRing
    if (k >= kRing && cudaStreamWaitEvent(c->pipe_in, c->ev_run[s], 0) != cudaSuccess) return SF_ECUDA;
    if (cudaMemcpyAsync(img, image, n * sizeof(float), cudaMemcpyHostToDevice, c->pipe_in) != cudaSuccess ||
        cudaMemcpyAsync(rng, range, n * sizeof(float), cudaMemcpyHostToDevice, c->pipe_in) != cudaSuccess ||
        cudaEventRecord(c->ev_in[s], c->pipe_in) != cudaSuccess)
        return SF_ECUDA;
    // the step: after its inputs, and after the slot's previous outputs left
    if (cudaStreamWaitEvent(st, c->ev_in[s], 0) != cudaSuccess ||
        (k >= kRing && cudaStreamWaitEvent(st, c->ev_out[s], 0) != cudaSuccess))
        return SF_ECUDA;
    const int r = sf_step(c, img, rng, dt, flow_out ? flow : nullptr, invdepth_out ? inv : nullptr, stream);
    if (r) return r;
    if (cudaEventRecord(c->ev_run[s], st) != cudaSuccess) return SF_ECUDA;
    // outputs
    if (cudaStreamWaitEvent(c->pipe_out, c->ev_run[s], 0) != cudaSuccess) return SF_ECUDA;
    if (flow_out && cudaMemcpyAsync(flow_out, flow, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, c->pipe_out) !=
                        cudaSuccess)
        return SF_ECUDA;
    if (invdepth_out &&
        cudaMemcpyAsync(invdepth_out, inv, n * sizeof(float), cudaMemcpyDeviceToHost, c->pipe_out) != cudaSuccess)
        return SF_ECUDA;
    if (cudaEventRecord(c->ev_out[s], c->pipe_out) != cudaSuccess ||
        cudaEventRecord(c->ev_done[k % kDone], c->pipe_out) != cudaSuccess)
        return SF_ECUDA;
    c->submitted = k + 1;
    if (ticket) *ticket = k;
    return SF_OK;
}

int sf_wait_host(sf_ctx* c, long long ticket)
{
    if (!c || ticket >= c->submitted || ticket < -1) return SF_EINVAL;
    if (ticket == -1) ticket = c->submitted - 1;
    if (ticket < 0) return SF_OK;   // nothing submitted
    // event ticket % kDone marks frame ticket while it is one of the last
    // kDone frames; an older ticket waits for the oldest of those instead
    // (output copies complete in submission order, so that implies its own)
    const long long w = std::max(ticket, c->submitted - kDone);
    return cudaEventSynchronize(c->ev_done[w % kDone]) == cudaSuccess ? SF_OK : SF_ECUDA;
}

int sf_status(sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    return engine_status(c->E);
}

int sf_get_state(sf_ctx* c, int level, float* dst, float* dt_prev, void* stream)
{
    if (!c || level < 0 || level >= c->E.st[0].L || !dst) return SF_EINVAL;
    sf_level_state& lv = c->E.st[0].lv[level];
    const int n = lv.grid.H * lv.grid.W;
    k_pack<<<std::min(ceil_div(n, 256), 1184), 256, 0, (cudaStream_t)stream>>>(lv.s0[c->E.parity],
                                                                              lv.s1[c->E.parity], dst, n);
    if (dt_prev) *dt_prev = c->E.dt_prev;
    return last_error();
}

int sf_set_state(sf_ctx* c, int level, const float* src, float dt_prev, void* stream)
{
    if (!c || level < 0 || level >= c->E.st[0].L || !src || !(dt_prev > 0.0f)) return SF_EINVAL;
    sf_level_state& lv = c->E.st[0].lv[level];
    const int n = lv.grid.H * lv.grid.W;
    k_unpack<<<std::min(ceil_div(n, 256), 1184), 256, 0, (cudaStream_t)stream>>>(src, lv.s0[c->E.parity],
                                                                                lv.s1[c->E.parity], n);
    c->E.dt_prev = dt_prev;
    c->E.initialised = 1;
    return last_error();
}

int sf_profile(sf_ctx* c, int enable)
{
    if (!c) return SF_EINVAL;
    c->E.prof.enabled = enable != 0;
    return SF_OK;
}

int sf_profile_read(sf_ctx* c, float* ms, int* count, int n)
{
    if (!c || (n > 0 && (!ms || !count))) return SF_EINVAL;
    const int r = c->E.prof.read(ms, count, n);
    if (r) return r;
    return c->E.launches_per_step();
}

int sf_kernels_per_step(const sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    return c->E.launches_per_step();
}

int sf_nf_max(const sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    return c->E.nf_max;
}

int sf_solve_tile(const sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    return c->E.solve_t;
}

int sf_update_mode(const sf_ctx* c)
{
    if (!c) return SF_EINVAL;
    return c->E.update_mode;
}

int sf_set_motion(sf_ctx* c, const float* omega, const float* accel, void* stream)
{
    if (!c) return SF_EINVAL;
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 3; ++k) {
        if (omega) m[k] = omega[k];
        if (accel) m[3 + k] = accel[k];
    }
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(m[k])) return SF_EINVAL;
    return cudaMemcpyAsync(c->E.st[0].motion, m, sizeof(m), cudaMemcpyHostToDevice, (cudaStream_t)stream) ==
                   cudaSuccess ? SF_OK : SF_ECUDA;
}

void sf_destroy(sf_ctx* c) { destroy_ctx(c); }

const char* sf_strerror(int code)
{
    switch (code) {
    case SF_OK: return "ok";
    case SF_EINVAL: return "invalid argument or configuration";
    case SF_ENOMEM: return "out of memory";
    case SF_ECUDA: return "CUDA runtime error";
    case SF_ETIMEOUT: return "bounded device wait timed out";
    case SF_ENONFINITE: return "non-finite value in the filter state";
    case SF_WARN_CFL: return "prediction violated the CFL bound (Eq. 67)";
    default: return "unknown status code";
    }
}

// ---------------------------------------------------------------------------
// C ABI: batched streams
// ---------------------------------------------------------------------------

int sf_batch_create(int n, const int* H, const int* W, const int* levels, const sf_params* params, sf_batch** out)
{
    if (out) *out = nullptr;
    if (n < 1 || n > 4096 || !H || !W || !levels || !params || !out) return SF_EINVAL;
    for (int s = 0; s < n; ++s) {
        const int r = check_params(H[s], W[s], levels[s], params + s);
        if (r) return r;
        if ((params[s].flags & (SF_DOMINANT_LITERAL | SF_SOURCE_SPLIT)) !=
            (params[0].flags & (SF_DOMINANT_LITERAL | SF_SOURCE_SPLIT)))
            return SF_EINVAL;   // one scheme variant per batch (one kernel instantiation)
    }
    sf_batch* b = new (std::nothrow) sf_batch();
    if (!b) return SF_ENOMEM;
    Engine& E = b->E;
    E.st.resize(n);
    E.flags = params[0].flags;
    E.nf_max = params[0].nf_max ? params[0].nf_max : kNfLimit;
    E.update_mode = params[0].update_mode ? params[0].update_mode : 1;
    E.update_auto = params[0].update_mode == 0 && (params[0].flags & SF_AUTOTUNE);
    size_t io_floats = 0;
    for (int s = 0; s < n; ++s) io_floats += 6 * (size_t)H[s] * W[s];   // image, range, flow (3), inverse depth
    int r = SF_OK;
    if (cudaMalloc(&E.io, io_floats * sizeof(float)) != cudaSuccess) { E.io = nullptr; r = SF_ENOMEM; }
    if (!r && cudaMemset(E.io, 0, io_floats * sizeof(float)) != cudaSuccess) r = SF_ECUDA;
    size_t off = 0;
    for (int s = 0; s < n && !r; ++s) {
        EngineStream& es = E.st[s];
        std::memset(&es, 0, sizeof(es));
        es.H = H[s]; es.W = W[s]; es.L = levels[s]; es.p = params[s];
        const size_t np = (size_t)H[s] * W[s];
        float* base = (float*)E.io + off;
        es.image = base; es.range = base + np; es.flow = base + 2 * np; es.inv = base + 5 * np;
        off += 6 * np;
    }
    if (!r) engine_solve_tile(E, params[0].solve_tile);
    if (!r) r = engine_init(E);
    if (r) { destroy_batch(b); return r; }
    *out = b;
    return SF_OK;
}

int sf_batch_buffers(sf_batch* b, int s, float** image, float** range, float** flow, float** invdepth)
{
    if (!b || s < 0 || s >= (int)b->E.st.size()) return SF_EINVAL;
    const EngineStream& es = b->E.st[s];
    if (image) *image = es.image;
    if (range) *range = es.range;
    if (flow) *flow = es.flow;
    if (invdepth) *invdepth = es.inv;
    return SF_OK;
}

int sf_batch_step(sf_batch* b, float dt, void* stream)
{
    if (!b || !(dt > 0.0f) || !std::isfinite(dt)) return SF_EINVAL;
    Engine& E = b->E;
    cudaStream_t st = (cudaStream_t)stream;
    const float wscale = E.initialised ? dt / E.dt_prev : 1.0f;   // reading R9
    const int q = E.parity;
    int r;
    // steady state (same dt as the previous frame, initialised, a capturable
    // stream, launch attributes already set by earlier plain steps, not
    // profiling): replay the frame's graph for this parity
    const bool graphable = E.initialised && wscale == 1.0f && st != nullptr && E.steps_plain >= 2 && !E.prof.enabled;
    if (graphable) {
        if (!E.graph[q] || E.graph_dt[q] != dt) {
            if (E.graph[q]) { cudaGraphExecDestroy(E.graph[q]); E.graph[q] = nullptr; }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SF_ECUDA;
            r = engine_launches(E, nullptr, nullptr, dt, 1.0f, nullptr, nullptr, st);
            const cudaError_t e = cudaStreamEndCapture(st, &g);
            if (r || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return r ? r : SF_ECUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&E.graph[q], g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) { E.graph[q] = nullptr; return SF_ECUDA; }
            E.graph_dt[q] = dt;
        }
        if (cudaGraphLaunch(E.graph[q], st) != cudaSuccess) return SF_ECUDA;
    } else {
        r = engine_launches(E, nullptr, nullptr, dt, wscale, nullptr, nullptr, st);
        if (r) return r;
        if (E.initialised) E.steps_plain++;
    }
    E.parity ^= 1;
    E.initialised = 1;
    E.dt_prev = dt;
    return SF_OK;
}

int sf_batch_status(sf_batch* b)
{
    if (!b) return SF_EINVAL;
    return engine_status(b->E);
}

int sf_batch_launches_per_step(const sf_batch* b)
{
    if (!b) return SF_EINVAL;
    return b->E.launches_per_step();
}

int sf_batch_nf_max(const sf_batch* b)
{
    if (!b) return SF_EINVAL;
    return b->E.nf_max;
}

int sf_batch_solve_tile(const sf_batch* b)
{
    if (!b) return SF_EINVAL;
    return b->E.solve_t;
}

int sf_batch_update_mode(const sf_batch* b)
{
    if (!b) return SF_EINVAL;
    return b->E.update_mode;
}

int sf_batch_motion(sf_batch* b, int s, float** motion)
{
    if (!b || !motion || s < 0 || s >= (int)b->E.st.size()) return SF_EINVAL;
    *motion = b->E.st[s].motion;
    return SF_OK;
}

int sf_batch_profile(sf_batch* b, int enable)
{
    if (!b) return SF_EINVAL;
    b->E.prof.enabled = enable != 0;
    return SF_OK;
}

int sf_batch_profile_read(sf_batch* b, float* ms, int* count, int n)
{
    if (!b || (n > 0 && (!ms || !count))) return SF_EINVAL;
    const int r = b->E.prof.read(ms, count, n);
    if (r) return r;
    return b->E.launches_per_step();
}

void sf_batch_destroy(sf_batch* b) { destroy_batch(b); }

// ---------------------------------------------------------------------------
// C ABI: stage entry points
// ---------------------------------------------------------------------------

namespace {

// sf_propagate / sf_propagate_imu: imu (host, 6 floats, frame units) or null
int stage_propagate(const sf_grid* g, int N, int flags, float wscale, const float* imu, const float* s0_in,
                    const float* s1_in, float* s0_out, float* s1_out, int* status, void* stream)
{
    if (!g || g->H < 1 || g->W < 1 || N < 1 || !s0_in || !s0_out) return SF_EINVAL;
    if ((s1_in == nullptr) != (s1_out == nullptr)) return SF_EINVAL;
    if (!aligned16(s0_in) || !aligned16(s0_out) || !aligned16(s1_in) || !aligned16(s1_out)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool c8 = s1_in != nullptr;
    const int nseg = ceil_div(N, kNfLimit);
    const size_t n = (size_t)g->H * g->W;
    float4* scratch = nullptr;
    if (nseg > 1) {
        if (cudaMallocAsync((void**)&scratch, (c8 ? 2 : 1) * n * sizeof(float4), st) != cudaSuccess) return SF_ENOMEM;
    }
    int r = SF_OK;
    const float4* in0 = (const float4*)s0_in;
    const float4* in1 = (const float4*)s1_in;
    for (int k = 0; k < nseg && !r; ++k) {
        const bool to_out = ((nseg - 1 - k) % 2) == 0;
        float4* o0 = to_out ? (float4*)s0_out : scratch;
        float4* o1 = c8 ? (to_out ? (float4*)s1_out : scratch + n) : nullptr;
        PropJob j;
        std::memset(&j, 0, sizeof(j));
        j.g = make_grid(*g);
        j.in0[0] = j.in0[1] = in0;
        j.in1[0] = j.in1[1] = in1;
        j.out0 = o0;
        j.out1 = o1;
        j.nf = N / nseg + (k < N % nseg ? 1 : 0);
        j.apply_wscale = k == 0;
        j.dt = 1.0f / (float)N;
        j.tiles_x = ceil_div(g->W, prop_tile(j.nf));
        std::vector<int4> work;
        add_tiles(work, 0, g->H, g->W, prop_tile(j.nf), prop_tile_h(j.nf, prop_warps(j.nf)));
        Plan pl;
        pl.c8 = c8;
        pl.nf = j.nf;
        pl.warps = prop_warps(j.nf);
        pl.smem = prop_smem_bytes(pl.warps);
        // the job, its work list and the motion travel through stream-ordered scratch
        void* mem = nullptr;
        const size_t woff = work_offset(sizeof(PropJob));
        const size_t moff = woff + work_offset(work.size() * sizeof(int4));
        const size_t bytes = moff + 8 * sizeof(float);
        if (cudaMallocAsync(&mem, bytes, st) != cudaSuccess) { r = SF_ENOMEM; break; }
        if (imu) j.motion = (const float*)((unsigned char*)mem + moff);
        std::vector<unsigned char> host(bytes, 0);
        std::memcpy(host.data(), &j, sizeof(PropJob));
        std::memcpy(host.data() + woff, work.data(), work.size() * sizeof(int4));
        if (imu) std::memcpy(host.data() + moff, imu, 6 * sizeof(float));
        r = cudaMemcpyAsync(mem, host.data(), bytes, cudaMemcpyHostToDevice, st) == cudaSuccess ? SF_OK : SF_ECUDA;
        if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;  // host buffer lifetime
        pl.jobs = mem;
        pl.work = (int4*)((unsigned char*)mem + woff);
        pl.nwork = (int)work.size();
        if (!r) r = launch_propagate(pl, 0, wscale, flags, status, st);
        cudaFreeAsync(mem, st);
        in0 = o0;
        in1 = o1;
    }
    if (scratch) cudaFreeAsync(scratch, st);
    return r;
}

}  // namespace

int sf_propagate(const sf_grid* g, int N, int flags, float wscale, const float* s0_in, const float* s1_in,
                 float* s0_out, float* s1_out, int* status, void* stream)
{
    return stage_propagate(g, N, flags, wscale, nullptr, s0_in, s1_in, s0_out, s1_out, status, stream);
}

int sf_propagate_imu(const sf_grid* g, int N, int flags, float wscale, const float* imu, const float* s0_in,
                     const float* s1_in, float* s0_out, float* s1_out, int* status, void* stream)
{
    if (!imu) return SF_EINVAL;
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(imu[k])) return SF_EINVAL;
    return stage_propagate(g, N, flags | SF_IMU, wscale, imu, s0_in, s1_in, s0_out, s1_out, status, stream);
}

int sf_update(const sf_grid* g, int level, int top, int S, int init, const float* gamma, float lambda_ref,
              const float* image, const float* range, int H1, int W1, const float* s0_cur, const float* s1_cur,
              const float* p0, const float* p1, float* s0_new, float* s1_new, float* diag, void* stream)
{
    if (!g || !gamma || !image || !range || !s0_new || !s1_new || level < 1 || level > kMaxLevelsDev || S < 0 ||
        S > 16 || g->H < 1 || g->W < 1)
        return SF_EINVAL;
    if ((g->H << (level - 1)) > H1 || (g->W << (level - 1)) > W1) return SF_EINVAL;
    if (!init && (!p0 || (top ? (!s0_cur || !s1_cur) : !p1))) return SF_EINVAL;
    if (!(gamma[4] > 0.0f) || !(gamma[3] >= 0.0f)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)g->H * g->W;
    SolveJob j;
    std::memset(&j, 0, sizeof(j));
    j.g = make_grid(*g);
    j.level = level;
    j.top = top != 0;
    j.g1 = gamma[0]; j.g2 = gamma[1]; j.g3 = gamma[2]; j.g4 = gamma[3]; j.g5 = gamma[4];
    j.inv45 = 1.0f / (j.g4 + j.g5);
    j.inv5 = 1.0f / j.g5;
    j.s0_cur[0] = j.s0_cur[1] = (const float4*)s0_cur;
    j.s1_cur[0] = j.s1_cur[1] = (const float4*)s1_cur;
    j.p0 = (const float4*)p0;
    j.p1 = (const float4*)p1;
    j.diag = diag;
    j.tiles_x = ceil_div(g->W, kSolveT);
    SmoothJob m;
    std::memset(&m, 0, sizeof(m));
    m.H = g->H;
    m.W = g->W;
    m.S = S;
    m.top = top != 0;
    m.s0_new[0] = m.s0_new[1] = (float4*)s0_new;
    m.s1_new[0] = m.s1_new[1] = (float4*)s1_new;
    m.tiles_x = ceil_div(g->W, kSmoothT);
    std::vector<int4> wsolve, wsmooth;
    add_tiles(wsolve, 0, g->H, g->W, kSolveT, kSolveT);
    add_tiles(wsmooth, 0, g->H, g->W, kSmoothT, kSmoothT);
    // one stream-ordered allocation: the solution and Y-hat planes, then the
    // two launch descriptors
    const size_t fields = n * sizeof(float4) + ((n * sizeof(float) + 255) & ~(size_t)255);
    const size_t o_js = fields, o_ws = o_js + work_offset(sizeof(SolveJob));
    const size_t o_jm = o_ws + work_offset(wsolve.size() * sizeof(int4)), o_wm = o_jm + work_offset(sizeof(SmoothJob));
    const size_t bytes = o_wm + wsmooth.size() * sizeof(int4);
    unsigned char* mem = nullptr;
    if (cudaMallocAsync((void**)&mem, bytes, st) != cudaSuccess) return SF_ENOMEM;
    j.x_out = (float4*)mem;
    j.y_out = (float*)(mem + n * sizeof(float4));
    m.x_in = j.x_out;
    m.y_in = j.y_out;
    std::vector<unsigned char> host(bytes - fields);
    std::memcpy(host.data() + (o_js - fields), &j, sizeof(SolveJob));
    std::memcpy(host.data() + (o_ws - fields), wsolve.data(), wsolve.size() * sizeof(int4));
    std::memcpy(host.data() + (o_jm - fields), &m, sizeof(SmoothJob));
    std::memcpy(host.data() + (o_wm - fields), wsmooth.data(), wsmooth.size() * sizeof(int4));
    int r = cudaMemcpyAsync(mem + fields, host.data(), host.size(), cudaMemcpyHostToDevice, st) == cudaSuccess
                ? SF_OK : SF_ECUDA;
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;  // host buffer lifetime
    UpdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = image; a.range = range; a.H1 = H1; a.W1 = W1; a.lambda_ref = lambda_ref;
    a.parity = 0;   // s*_cur[0]; the smoothing writes slot q = 0 (both slots are the caller's planes)
    a.init = init != 0;
    Plan ps, pm;
    ps.jobs = mem + o_js; ps.work = (int4*)(mem + o_ws); ps.nwork = (int)wsolve.size();
    pm.jobs = mem + o_jm; pm.work = (int4*)(mem + o_wm); pm.nwork = (int)wsmooth.size(); pm.smem = smooth_smem_bytes(S);
    if (!r) r = launch_solve(ps, a, st);
    if (!r) r = launch_smooth(pm, 0, 1.0f, 0, nullptr, nullptr, nullptr, st);
    cudaFreeAsync(mem, st);
    return r;
}

namespace {

int remap_launch(int mode, const sf_grid* dst, const float* R, int Hs, int Ws, const float* cam,
                 const float* src_image, const float* src_range, float* out_image, float* out_range, void* stream)
{
    if (!dst || dst->H < 1 || dst->W < 1 || !R || Hs < 1 || Ws < 1 || !src_image || !out_image) return SF_EINVAL;
    if ((src_range == nullptr) != (out_range == nullptr)) return SF_EINVAL;
    if (!(dst->fx > 0) || !(dst->fy > 0) || !std::isfinite(dst->fx) || !std::isfinite(dst->fy) ||
        !std::isfinite(dst->cx) || !std::isfinite(dst->cy))
        return SF_EINVAL;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(R[k])) return SF_EINVAL;
    RemapArgs a;
    std::memset(&a, 0, sizeof(a));
    if (mode == 0) {
        if (!cam || !(cam[0] > 0) || !(cam[1] > 0)) return SF_EINVAL;
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(cam[k])) return SF_EINVAL;
        a.cfx = cam[0]; a.cfy = cam[1]; a.ccx = cam[2]; a.ccy = cam[3];
    }
    const Grid g = make_grid(*dst);
    a.H = dst->H; a.W = dst->W;
    a.gax = g.ax; a.gbx = g.bx; a.gay = g.ay; a.gby = g.by;
    for (int k = 0; k < 9; ++k) a.R[k] = R[k];
    a.Hs = Hs; a.Ws = Ws;
    a.img = src_image; a.rng = src_range;
    a.out_img = out_image; a.out_rng = out_range;
    const dim3 block(kRemapTX, kRemapTY), grid(ceil_div(dst->W, kRemapTX), ceil_div(dst->H, kRemapTY));
    if (mode == 0) k_remap<0><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    else k_remap<1><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    return last_error();
}

}  // namespace

int sf_remap_pinhole(const sf_grid* dst, const float* R, int Hs, int Ws, const float* cam, const float* src_image,
                     const float* src_range, float* out_image, float* out_range, void* stream)
{
    return remap_launch(0, dst, R, Hs, Ws, cam, src_image, src_range, out_image, out_range, stream);
}

int sf_remap_equirect(const sf_grid* dst, const float* R, int Hs, int Ws, const float* src_image,
                      const float* src_range, float* out_image, float* out_range, void* stream)
{
    return remap_launch(1, dst, R, Hs, Ws, nullptr, src_image, src_range, out_image, out_range, stream);
}

}  // extern "C"

namespace {

// The TMA description of an NHWC bf16 input for the convolution: dimensions
// (C, W, H, N) innermost first, boxes of 8 channels x kConvSlots pixels x 1 row
// x 1 image, zero fill outside the tensor.  cuTensorMapEncodeTiled comes from
// the driver through the runtime's entry-point query (no link to the driver
// library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int conv_input_map(const void* x, int N, int H, int W, int Cin, CUtensorMap* out)
{
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!fn) {
            void* p = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
                return SF_ECUDA;
            fn = (EncodeTiledFn)p;
        }
    }
    const cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)kConvSlots, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SF_OK : SF_ECUDA;
}

// strips of up to 32 output rows, shorter when that leaves fewer than three
// per SM (three CTAs fit an SM)
int conv_strip(int N, int H, int tiles_x)
{
    const int columns = N * tiles_x;
    return std::max(1, std::min(kConvStrip, ceil_div(H, std::max(1, ceil_div(kSmCount * 3, columns)))));
}

}  // namespace

extern "C" {

int sf_conv3x3(int N, int H, int W, int Cin, int Cout, const void* x, const void* w, const float* bias, int relu,
               void* y, float* y32, int* status, void* stream)
{
    if (N < 1 || H < 1 || W < 1 || (Cin != 16 && Cin != 32) || (Cout != 16 && Cout != 32) || !x || !w ||
        (!y && !y32))
        return SF_EINVAL;
    if (!aligned16(x) || !aligned16(w) || !aligned16(y) || !aligned16(y32)) return SF_EINVAL;
    if ((double)N * H * W * (Cin > Cout ? Cin : Cout) > 2147483647.0) return SF_EINVAL;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.N = N; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout;
    a.x = (const __nv_bfloat16*)x;
    a.w = (const __nv_bfloat16*)w;
    a.bias = bias;
    a.relu = relu != 0;
    a.y = (__nv_bfloat16*)y;
    a.y32 = y32;
    a.tiles_x = ceil_div(W, kConvM);
    a.n_tiles = N * H * a.tiles_x;
    a.status = status;
    a.spin_limit = kConvSpinLimit;
    a.strip = conv_strip(N, H, a.tiles_x);
    CUtensorMap map;
    if (conv_input_map(x, N, H, W, Cin, &map)) return SF_ECUDA;
    const size_t smem = conv_ws_smem_bytes(Cin, Cout);
    if (set_smem_attr((const void*)k_conv3x3, smem)) return SF_ECUDA;
    const int strips = N * a.tiles_x * ceil_div(H, a.strip);
    k_conv3x3<<<std::min(strips, kSmCount * 3), kConvWsThreads, smem, (cudaStream_t)stream>>>(map, a);
    return last_error();
}

// ---------------------------------------------------------------------------
// C ABI: the learned propagation surrogate
// ---------------------------------------------------------------------------

struct sf_surrogate {
    static constexpr int kL = 4;
    const int cin[kL] = {kSurrIn, kSurrHidden, kSurrHidden, kSurrHidden};
    const int cout[kL] = {kSurrHidden, kSurrHidden, kSurrHidden, kSurrOut};
    // parameters and optimiser state: per layer w (9 cout cin) then b (cout)
    float* param = nullptr;     // FP32 master copy
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    size_t off[kL + 1] = {};
    __nv_bfloat16* w16[kL] = {};
    __nv_bfloat16* w16t[kL] = {};
    void* wblock = nullptr;
    // activations, sized for cap pixels
    size_t cap = 0;
    void* ablock = nullptr;
    __nv_bfloat16 *x0 = nullptr, *a[3] = {}, *dy = nullptr, *dA = nullptr, *dB = nullptr;
    float* y32 = nullptr;
    float* loss = nullptr;
    int* status = nullptr;
    int steps = 0;
};

namespace {

inline size_t layer_params(int cin, int cout) { return (size_t)9 * cin * cout + cout; }

void surrogate_free(sf_surrogate* s)
{
    if (!s) return;
    cudaFree(s->wblock);
    cudaFree(s->ablock);
    delete s;
}

int surrogate_capacity(sf_surrogate* s, size_t px)
{
    if (px <= s->cap) return SF_OK;
    cudaFree(s->ablock);
    s->ablock = nullptr;
    s->cap = 0;
    const size_t b16 = px * 2;   // bytes per channel (bf16)
    const size_t bytes = b16 * kSurrIn + 3 * b16 * kSurrHidden + b16 * kSurrOut + 2 * b16 * kSurrHidden +
                         px * kSurrOut * sizeof(float) + 256;
    if (cudaMalloc(&s->ablock, bytes) != cudaSuccess) { s->ablock = nullptr; return SF_ENOMEM; }
    unsigned char* p = (unsigned char*)s->ablock;
    auto take = [&](size_t n) { unsigned char* q = p; p += (n + 255) & ~(size_t)255; return q; };
    s->x0 = (__nv_bfloat16*)take(b16 * kSurrIn);
    for (int k = 0; k < 3; ++k) s->a[k] = (__nv_bfloat16*)take(b16 * kSurrHidden);
    s->dy = (__nv_bfloat16*)take(b16 * kSurrOut);
    s->dA = (__nv_bfloat16*)take(b16 * kSurrHidden);
    s->dB = (__nv_bfloat16*)take(b16 * kSurrHidden);
    s->y32 = (float*)take(px * kSurrOut * sizeof(float));
    s->cap = px;
    return SF_OK;
}

int conv_launch(const sf_surrogate* s, int N, int H, int W, int cin, int cout, const __nv_bfloat16* x,
                const __nv_bfloat16* w, const float* b, int relu, __nv_bfloat16* y, float* y32, cudaStream_t st)
{
    return sf_conv3x3(N, H, W, cin, cout, x, w, b, relu, y, y32, s->status, st);
}

inline int grid_stride_blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, kSmCount * 8); }


// weight and bias gradients of one 3x3 layer, ADDED into dw [9][Cout][Cin]
// and db [Cout] (the caller zeroes them)
int wgrad_launch(int N, int H, int W, int Cin, int Cout, const __nv_bfloat16* x, const __nv_bfloat16* dy, float* dw,
                 float* db, cudaStream_t st, int* status = nullptr)
{
    WgradArgs a;
    std::memset(&a, 0, sizeof(a));
    a.N = N; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout;
    a.x = x; a.dy = dy; a.dw = dw; a.db = db;
    a.tiles_x = ceil_div(W, kConvM);
    a.spin_limit = kConvSpinLimit;
    a.status = status;
    // strips of up to 32 rows, shorter when that leaves fewer than 2 per SM
    const int columns = N * a.tiles_x;
    a.strip = std::max(1, std::min(kConvStrip, ceil_div(H, std::max(1, ceil_div(kSmCount * 2, columns)))));
    const int strips = columns * ceil_div(H, a.strip);
    const size_t smem = wgrad_tc_smem_bytes();
    if (set_smem_attr((const void*)k_wgrad_tc, smem)) return SF_ECUDA;
    k_wgrad_tc<<<std::min(strips, kSmCount * 2), kWgtThreads, smem, st>>>(a);
    return last_error();
}

// features, the four layers (the three hidden activations kept for the
// backward pass), FP32 output in y32
int surrogate_forward(sf_surrogate* s, const Grid& g, int n, const float4* s0, cudaStream_t st)
{
    const size_t px = (size_t)n * g.H * g.W;
    k_surr_features<<<grid_stride_blocks(px), 256, 0, st>>>(g, n, s0, s->x0);
    int r = last_error();
    const __nv_bfloat16* in = s->x0;
    for (int l = 0; l < 3 && !r; ++l) {
        r = conv_launch(s, n, g.H, g.W, s->cin[l], s->cout[l], in, s->w16[l], s->param + s->off[l] + 9 * s->cin[l] *
                        s->cout[l], 1, s->a[l], nullptr, st);
        in = s->a[l];
    }
    if (!r)
        r = conv_launch(s, n, g.H, g.W, s->cin[3], s->cout[3], in, s->w16[3],
                        s->param + s->off[3] + 9 * s->cin[3] * s->cout[3], 0, nullptr, s->y32, st);
    return r;
}

extern "C++" {   // an internal helper, declared ahead of the engine code
// the features, the whole network and the head in one launch (k_surr_net)
// for n <= kNetMaxImg images of one grid whose states are separate planes
// s0[k] -> p0[k]: strips of kNetStrip output rows, halved while the launch
// would still fill at most half the SMs (down to 16); one CTA per SM walks
// the units.  Measured on 16 frames of 1024 x 1024: strips of 64, 128 and
// 256 rows ran 2.31, 2.21 and 2.16 ms (the features then a launch of their own).
int net_forward(sf_surrogate* s, const Grid& g, int n, const float4* const* s0, float4* const* p0, cudaStream_t st)
{
    if (n < 1 || n > kNetMaxImg) return SF_EINVAL;
    NetArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.N = n;
    for (int k = 0; k < n; ++k) { a.s0[k] = s0[k]; a.p0[k] = p0[k]; }
    for (int l = 0; l < sf_surrogate::kL; ++l) {
        a.w16[l] = s->w16[l];
        a.bias[l] = s->param + s->off[l] + 9 * s->cin[l] * s->cout[l];
    }
    a.tiles_x = ceil_div(g.W, kNetValid);
    a.spin_limit = kConvSpinLimit;
    a.status = s->status;
    a.strip = kNetStrip;
    auto units = [&](int strip) { return (long)n * a.tiles_x * ceil_div(g.H, strip); };
    while (a.strip > 16 && units(a.strip) * 2 <= kSmCount) a.strip /= 2;
    if (set_smem_attr((const void*)k_surr_net, net_smem_bytes())) return SF_ECUDA;
    k_surr_net<<<(int)std::min<long>(units(a.strip), kSmCount), kNetThreads, net_smem_bytes(), st>>>(a);
    return last_error();
}
}  // extern "C++"

}  // namespace

int sf_conv3x3_wgrad(int N, int H, int W, int Cin, int Cout, const void* x, const void* dy, float* dw, float* db,
                     void* stream)
{
    if (N < 1 || H < 1 || W < 1 || (Cin != 16 && Cin != 32) || (Cout != 16 && Cout != 32) || !x || !dy || !dw ||
        !db)
        return SF_EINVAL;
    if (!aligned16(x) || !aligned16(dy) || !aligned16(dw) || !aligned16(db)) return SF_EINVAL;
    if ((double)N * H * W * (Cin > Cout ? Cin : Cout) > 2147483647.0) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // the kernel adds into its outputs
    if (cudaMemsetAsync(dw, 0, (size_t)9 * Cin * Cout * sizeof(float), st) != cudaSuccess) return SF_ECUDA;
    if (cudaMemsetAsync(db, 0, (size_t)Cout * sizeof(float), st) != cudaSuccess) return SF_ECUDA;
    return wgrad_launch(N, H, W, Cin, Cout, (const __nv_bfloat16*)x, (const __nv_bfloat16*)dy, dw, db, st);
}

int sf_selftest_conv_timeout(void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    // one tile: 1 x 1 x 128 pixels, 16 -> 16 channels, zero data
    const size_t xb = 128 * 16 * 2, wb = 9 * 16 * 16 * 2, yb = 128 * 16 * 2;
    unsigned char* mem = nullptr;
    if (cudaMallocAsync((void**)&mem, xb + wb + yb + 256, st) != cudaSuccess) return SF_ENOMEM;
    int r = cudaMemsetAsync(mem, 0, xb + wb + yb + 256, st) == cudaSuccess ? SF_OK : SF_ECUDA;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.N = 1; a.H = 1; a.W = 128; a.Cin = 16; a.Cout = 16;
    a.x = (const __nv_bfloat16*)mem;
    a.w = (const __nv_bfloat16*)(mem + xb);
    a.y = (__nv_bfloat16*)(mem + xb + wb);
    a.tiles_x = 1; a.n_tiles = 1; a.strip = 1;
    a.status = (int*)(mem + xb + wb + yb);
    a.spin_limit = 1024;      // a short limit: the test ends in well under a second
    a.no_commit = 1;          // nothing is issued, so the wait cannot complete
    CUtensorMap map;
    if (!r && conv_input_map(a.x, 1, 1, 128, 16, &map)) r = SF_ECUDA;
    if (!r && set_smem_attr((const void*)k_conv3x3, conv_ws_smem_bytes(16, 16))) r = SF_ECUDA;
    if (!r) {
        k_conv3x3<<<1, kConvWsThreads, conv_ws_smem_bytes(16, 16), st>>>(map, a);
        r = last_error();
    }
    int s = 0;
    if (!r) r = cudaMemcpyAsync(&s, a.status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess ? SF_OK : SF_ECUDA;
    cudaFreeAsync(mem, st);
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (r) return r;
    return (s & kStatusTimeout) ? SF_ETIMEOUT : SF_OK;
}

int sf_selftest_net_timeout(void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    // one 16 x 16 frame, zero state and weights; the MMA thread issues nothing
    const int H = 16, W = 16;
    const size_t sb = (size_t)H * W * sizeof(float4);
    const size_t wb = (size_t)(kNetW1 + 2 * kNetW2 + kNetW4);   // bytes of the four layers' BF16 weights
    unsigned char* mem = nullptr;
    if (cudaMallocAsync((void**)&mem, 2 * sb + wb + 256, st) != cudaSuccess) return SF_ENOMEM;
    int r = cudaMemsetAsync(mem, 0, 2 * sb + wb + 256, st) == cudaSuccess ? SF_OK : SF_ECUDA;
    sf_grid sg;
    std::memset(&sg, 0, sizeof(sg));
    sg.H = H; sg.W = W; sg.fx = sg.fy = 8.0f; sg.cx = sg.cy = 8.0f;
    NetArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = make_grid(sg);
    a.N = 1;
    a.s0[0] = (const float4*)mem;
    a.p0[0] = (float4*)(mem + sb);
    a.w16[0] = (const __nv_bfloat16*)(mem + 2 * sb);
    a.w16[1] = (const __nv_bfloat16*)(mem + 2 * sb + kNetW1);
    a.w16[2] = (const __nv_bfloat16*)(mem + 2 * sb + kNetW1 + kNetW2);
    a.w16[3] = (const __nv_bfloat16*)(mem + 2 * sb + kNetW1 + 2 * kNetW2);
    a.tiles_x = 1;
    a.strip = H;
    a.status = (int*)(mem + 2 * sb + wb);
    a.spin_limit = 1024;      // a short limit: the test ends in well under a second
    a.no_commit = 1;          // nothing is issued, so the waits cannot complete
    if (!r && set_smem_attr((const void*)k_surr_net, net_smem_bytes())) r = SF_ECUDA;
    if (!r) {
        k_surr_net<<<1, kNetThreads, net_smem_bytes(), st>>>(a);
        r = last_error();
    }
    int s = 0;
    if (!r) r = cudaMemcpyAsync(&s, a.status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess ? SF_OK : SF_ECUDA;
    cudaFreeAsync(mem, st);
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (r) return r;
    return (s & kStatusTimeout) ? SF_ETIMEOUT : SF_OK;
}

int sf_surrogate_create(unsigned long long seed, sf_surrogate** out)
{
    if (!out) return SF_EINVAL;
    *out = nullptr;
    sf_surrogate* s = new (std::nothrow) sf_surrogate();
    if (!s) return SF_ENOMEM;
    for (int l = 0; l < sf_surrogate::kL; ++l) s->off[l + 1] = s->off[l] + layer_params(s->cin[l], s->cout[l]);
    const size_t np = s->off[sf_surrogate::kL];
    size_t n16 = 0;
    for (int l = 0; l < sf_surrogate::kL; ++l) n16 += 9 * (size_t)s->cin[l] * s->cout[l];
    const size_t bytes = 4 * np * sizeof(float) + 2 * n16 * sizeof(__nv_bfloat16) + 2 * sizeof(float) + 256 * 12;
    if (cudaMalloc(&s->wblock, bytes) != cudaSuccess) { s->wblock = nullptr; surrogate_free(s); return SF_ENOMEM; }
    unsigned char* p = (unsigned char*)s->wblock;
    auto take = [&](size_t nb) { unsigned char* q = p; p += (nb + 255) & ~(size_t)255; return q; };
    s->param = (float*)take(np * sizeof(float));
    s->grad = (float*)take(np * sizeof(float));
    s->m1 = (float*)take(np * sizeof(float));
    s->m2 = (float*)take(np * sizeof(float));
    for (int l = 0; l < sf_surrogate::kL; ++l) {
        s->w16[l] = (__nv_bfloat16*)take(9 * (size_t)s->cin[l] * s->cout[l] * 2);
        s->w16t[l] = (__nv_bfloat16*)take(9 * (size_t)s->cin[l] * s->cout[l] * 2);
    }
    s->loss = (float*)take(sizeof(float));
    s->status = (int*)take(sizeof(int));
    // He-normal weights over the used inputs, zero biases, a small last layer
    // (the untrained network predicts nearly no change)
    std::vector<float> h(np, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    const int used_in[sf_surrogate::kL] = {6, kSurrHidden, kSurrHidden, kSurrHidden};
    for (int l = 0; l < sf_surrogate::kL; ++l) {
        const float sd = std::sqrt(2.0f / (9.0f * used_in[l])) * (l == sf_surrogate::kL - 1 ? 0.1f : 1.0f);
        for (size_t k = 0; k < 9 * (size_t)s->cin[l] * s->cout[l]; ++k) {
            const int ci = (int)(k % s->cin[l]);
            h[s->off[l] + k] = ci < used_in[l] ? sd * nd(rng) : 0.0f;
        }
    }
    int r = cudaMemcpy(s->param, h.data(), np * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) r = cudaMemset(s->m1, 0, np * sizeof(float)) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) r = cudaMemset(s->m2, 0, np * sizeof(float)) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) r = cudaMemset(s->status, 0, sizeof(int)) == cudaSuccess ? SF_OK : SF_ECUDA;
    for (int l = 0; l < sf_surrogate::kL && !r; ++l) {
        k_weights_bf16<<<64, 256>>>(s->cin[l], s->cout[l], s->param + s->off[l], s->w16[l], s->w16t[l]);
        r = last_error();
    }
    if (!r) r = cudaDeviceSynchronize() == cudaSuccess ? SF_OK : SF_ECUDA;
    if (r) { surrogate_free(s); return r; }
    *out = s;
    return SF_OK;
}

void sf_surrogate_destroy(sf_surrogate* s) { surrogate_free(s); }

int sf_surrogate_num_params(const sf_surrogate* s)
{
    if (!s) return SF_EINVAL;
    return (int)s->off[sf_surrogate::kL];
}

int sf_surrogate_params(sf_surrogate* s, float* host, int set)
{
    if (!s || !host) return SF_EINVAL;
    const size_t np = s->off[sf_surrogate::kL];
    if (!set) return cudaMemcpy(host, s->param, np * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? SF_OK : SF_ECUDA;
    for (size_t k = 0; k < np; ++k)
        if (!std::isfinite(host[k])) return SF_EINVAL;
    if (cudaMemcpy(s->param, host, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return SF_ECUDA;
    for (int l = 0; l < sf_surrogate::kL; ++l) {
        k_weights_bf16<<<64, 256>>>(s->cin[l], s->cout[l], s->param + s->off[l], s->w16[l], s->w16t[l]);
        if (last_error()) return SF_ECUDA;
    }
    return cudaDeviceSynchronize() == cudaSuccess ? SF_OK : SF_ECUDA;
}

int sf_surrogate_forward_layered(sf_surrogate* s, const sf_grid* g, int n, const float* s0, float* p0, void* stream)
{
    if (!s || !g || g->H < 1 || g->W < 1 || n < 1 || !s0 || !p0 || !aligned16(s0) || !aligned16(p0)) return SF_EINVAL;
    const size_t px = (size_t)n * g->H * g->W;
    if (px * kSurrHidden > 2147483647ull) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int r = surrogate_capacity(s, px);
    const Grid gg = make_grid(*g);
    if (!r) r = surrogate_forward(s, gg, n, (const float4*)s0, st);
    if (!r) {
        k_surr_head<<<grid_stride_blocks(px), 256, 0, st>>>(gg, n, (const float4*)s0, s->y32, (float4*)p0);
        r = last_error();
    }
    return r;
}

int sf_surrogate_forward(sf_surrogate* s, const sf_grid* g, int n, const float* s0, float* p0, void* stream)
{
    if (!s || !g || g->H < 1 || g->W < 1 || n < 1 || !s0 || !p0 || !aligned16(s0) || !aligned16(p0)) return SF_EINVAL;
    const size_t px = (size_t)n * g->H * g->W;
    if (px * kSurrHidden > 2147483647ull) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const Grid gg = make_grid(*g);
    const size_t hw = (size_t)g->H * g->W;
    int r = SF_OK;
    for (int k0 = 0; k0 < n && !r; k0 += kNetMaxImg) {            // kNetMaxImg images per launch
        const int m = std::min(kNetMaxImg, n - k0);
        const float4* in[kNetMaxImg];
        float4* out[kNetMaxImg];
        for (int k = 0; k < m; ++k) {
            in[k] = (const float4*)s0 + (size_t)(k0 + k) * hw;
            out[k] = (float4*)p0 + (size_t)(k0 + k) * hw;
        }
        r = net_forward(s, gg, m, in, out, st);
    }
    return r;
}

int sf_surrogate_train_step(sf_surrogate* s, const sf_grid* g, int n, const float* s0, const float* target, float lr,
                            float* loss_out, void* stream)
{
    if (!s || !g || g->H < 1 || g->W < 1 || n < 1 || !s0 || !target || !aligned16(s0) || !aligned16(target) ||
        !(lr >= 0.0f) || !std::isfinite(lr))
        return SF_EINVAL;
    const size_t px = (size_t)n * g->H * g->W;
    if (px * kSurrHidden > 2147483647ull) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int r = surrogate_capacity(s, px);
    const Grid gg = make_grid(*g);
    const size_t np = s->off[sf_surrogate::kL];
    if (!r) r = surrogate_forward(s, gg, n, (const float4*)s0, st);
    if (!r) r = cudaMemsetAsync(s->loss, 0, sizeof(float), st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) r = cudaMemsetAsync(s->grad, 0, np * sizeof(float), st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (!r) {
        k_surr_loss_grad<<<grid_stride_blocks(px), 256, 0, st>>>(gg, n, (const float4*)s0, (const float4*)target,
                                                                   s->y32, s->dy, 1.0f / (4.0f * (float)px), s->loss);
        r = last_error();
    }
    // backward: dy of layer l is `d`, its input activation `in`
    const __nv_bfloat16* d = s->dy;
    __nv_bfloat16* bufs[2] = {s->dA, s->dB};
    for (int l = sf_surrogate::kL - 1; l >= 0 && !r; --l) {
        const __nv_bfloat16* in = l == 0 ? s->x0 : s->a[l - 1];
        r = wgrad_launch(n, g->H, g->W, s->cin[l], s->cout[l], in, d, s->grad + s->off[l],
                         s->grad + s->off[l] + 9 * s->cin[l] * s->cout[l], st, s->status);
        if (r || l == 0) break;
        __nv_bfloat16* dx = bufs[l & 1];
        r = conv_launch(s, n, g->H, g->W, s->cout[l], s->cin[l], d, s->w16t[l], nullptr, 0, dx, nullptr, st);
        if (r) break;
        k_relu_mask<<<grid_stride_blocks(px * s->cin[l]), 256, 0, st>>>(px * s->cin[l], dx, s->a[l - 1]);
        r = last_error();
        d = dx;
    }
    // Adam
    if (!r) {
        s->steps++;
        AdamArgs h;
        h.lr = lr; h.beta1 = 0.9f; h.beta2 = 0.999f; h.eps = 1e-8f;
        h.c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)s->steps)));
        h.c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)s->steps)));
        for (int l = 0; l < sf_surrogate::kL && !r; ++l) {
            const size_t nw = 9 * (size_t)s->cin[l] * s->cout[l];
            float* base = s->param + s->off[l];
            k_adam_layer<<<64, 256, 0, st>>>(s->cin[l], s->cout[l], h, base, s->grad + s->off[l], s->m1 + s->off[l],
                                             s->m2 + s->off[l], base + nw, s->grad + s->off[l] + nw,
                                             s->m1 + s->off[l] + nw, s->m2 + s->off[l] + nw, s->w16[l], s->w16t[l]);
            r = last_error();
        }
    }
    if (!r && loss_out) {
        float sum = 0.0f;
        r = cudaMemcpyAsync(&sum, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st) == cudaSuccess ? SF_OK : SF_ECUDA;
        if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
        *loss_out = sum / (4.0f * (float)px);
    }
    if (!r) {
        int stv = 0;
        if (cudaMemcpyAsync(&stv, s->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SF_ECUDA;
        if (stv & kStatusTimeout) return SF_ETIMEOUT;
    }
    return r;
}

int sf_surrogate_propagate(sf_surrogate* s, const sf_grid* g, int n, int N, const float* s0, float* p0,
                           float threshold_px, float* residual_px, int* used_plain, void* stream)
{
    if (!s || !g || g->H < 1 || g->W < 1 || n < 1 || N < 1 || !s0 || !p0 || !aligned16(s0) || !aligned16(p0) ||
        !(threshold_px >= 0.0f))
        return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t px = (size_t)n * g->H * g->W;
    const Grid gg = make_grid(*g);
    // the surrogate's prediction, then one plain step (N = 1) of every frame
    int r = sf_surrogate_forward(s, g, n, s0, p0, stream);
    float4* one = nullptr;
    unsigned* dmax = nullptr;
    if (!r && cudaMallocAsync((void**)&one, px * sizeof(float4) + 256, st) != cudaSuccess) r = SF_ENOMEM;
    if (!r) {
        dmax = (unsigned*)(one + px);
        r = cudaMemsetAsync(dmax, 0, sizeof(unsigned), st) == cudaSuccess ? SF_OK : SF_ECUDA;
    }
    const size_t frame = (size_t)g->H * g->W;
    for (int k = 0; k < n && !r; ++k)
        r = sf_propagate(g, 1, 0, 1.0f, s0 + 4 * frame * k, nullptr, (float*)(one + frame * k), nullptr, nullptr, stream);
    if (!r) {
        k_surr_maxdiff<<<grid_stride_blocks(px), 256, 0, st>>>(gg, n, (const float4*)p0, one, dmax);
        r = last_error();
    }
    unsigned bits = 0;
    if (!r) r = cudaMemcpyAsync(&bits, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (one) cudaFreeAsync(one, st);
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
    if (r) return r;
    float res;
    std::memcpy(&res, &bits, sizeof(res));
    if (residual_px) *residual_px = res;
    const int fallback = !(res <= threshold_px);
    if (used_plain) *used_plain = fallback;
    // the fallback: the plain propagation with the full N sub-iterations
    for (int k = 0; k < n && fallback && !r; ++k)
        r = sf_propagate(g, N, 0, 1.0f, s0 + 4 * frame * k, nullptr, p0 + 4 * frame * k, nullptr, nullptr, stream);
    return r;
}

namespace {

// attach (or detach, s = null) a surrogate for every stream's top level
int engine_attach(Engine& E, sf_surrogate* s)
{
    int r = SF_OK;
    if (s) {
        bool same = true;
        const sf_grid& g0 = E.st[0].lv[E.st[0].L - 1].grid;
        for (auto& es : E.st) {
            const sf_grid& gt = es.lv[es.L - 1].grid;
            same = same && gt.H == g0.H && gt.W == g0.W && gt.fx == g0.fx && gt.fy == g0.fy && gt.cx == g0.cx &&
                   gt.cy == g0.cy;
        }
        E.surr_same_grid = same;
        // the kernels' shared-memory limits are raised here, outside any stream capture
        if (set_smem_attr((const void*)k_surr_net, net_smem_bytes())) r = SF_ECUDA;
        if (!r && set_smem_attr((const void*)k_conv3x3, conv_ws_smem_bytes(kSurrHidden, kSurrHidden))) r = SF_ECUDA;
        if (r) return r;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SF_ECUDA;
    E.surr = s;
    r = engine_prop_plans(E, st);
    if (!r) r = cudaStreamSynchronize(st) == cudaSuccess ? SF_OK : SF_ECUDA;
    cudaStreamDestroy(st);
    for (int q = 0; q < 2; ++q)
        if (E.graph[q]) { cudaGraphExecDestroy(E.graph[q]); E.graph[q] = nullptr; }
    E.steps_plain = 0;
    return r;
}

}  // namespace

int sf_set_surrogate(sf_ctx* c, sf_surrogate* s)
{
    if (!c) return SF_EINVAL;
    return engine_attach(c->E, s);
}

int sf_batch_set_surrogate(sf_batch* b, sf_surrogate* s)
{
    if (!b) return SF_EINVAL;
    return engine_attach(b->E, s);
}

namespace {

// threshold of stream s (-1: every stream, and streams attached later)
int engine_surr_threshold(Engine& E, int s, float thr)
{
    if (!(thr >= 0.0f)) return SF_EINVAL;   // NaN or negative; +inf: never fall back
    const int n = (int)E.st.size();
    if (s < -1 || s >= n) return SF_EINVAL;
    if (s == -1) E.surr_thr_default = thr;
    if (!E.surr_thr) return s == -1 ? SF_OK : SF_EINVAL;   // no surrogate attached yet
    std::vector<float> v(s == -1 ? n : 1, thr);
    return cudaMemcpy(E.surr_thr + (s == -1 ? 0 : s), v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice) ==
                   cudaSuccess ? SF_OK : SF_ECUDA;
}

int engine_surr_stats(Engine& E, float* residual_px, int* fallbacks, int n)
{
    if (n < 1 || n > (int)E.st.size() || (!residual_px && !fallbacks)) return SF_EINVAL;
    if (!E.surr_res) return SF_EINVAL;                     // never attached
    if (cudaDeviceSynchronize() != cudaSuccess) return SF_ECUDA;
    std::vector<unsigned> r(n), c(n);
    if (cudaMemcpy(r.data(), E.surr_res, n * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(c.data(), E.surr_cnt, n * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SF_ECUDA;
    for (int k = 0; k < n; ++k) {
        if (residual_px) std::memcpy(residual_px + k, &r[k], sizeof(float));
        if (fallbacks) fallbacks[k] = (int)c[k];
    }
    return SF_OK;
}

}  // namespace

int sf_set_trace(int enable)
{
    g_trace.store(enable != 0, std::memory_order_relaxed);
    return SF_OK;
}

int sf_set_surrogate_threshold(sf_ctx* c, float threshold_px)
{
    if (!c) return SF_EINVAL;
    return engine_surr_threshold(c->E, -1, threshold_px);
}

int sf_batch_set_surrogate_threshold(sf_batch* b, int s, float threshold_px)
{
    if (!b) return SF_EINVAL;
    return engine_surr_threshold(b->E, s, threshold_px);
}

int sf_surrogate_stats(sf_ctx* c, float* residual_px, int* fallbacks)
{
    if (!c) return SF_EINVAL;
    return engine_surr_stats(c->E, residual_px, fallbacks, 1);
}

int sf_batch_surrogate_stats(sf_batch* b, float* residual_px, int* fallbacks, int n)
{
    if (!b) return SF_EINVAL;
    return engine_surr_stats(b->E, residual_px, fallbacks, n);
}

int sf_surrogate_grads(sf_surrogate* s, float* host)
{
    if (!s || !host) return SF_EINVAL;
    return cudaMemcpy(host, s->grad, s->off[sf_surrogate::kL] * sizeof(float), cudaMemcpyDeviceToHost) ==
                   cudaSuccess ? SF_OK : SF_ECUDA;
}

int sf_reconstruct(int levels, const sf_grid* grids, float* const* s0, const float* const* s1, float dt,
                   float* flow_out, float* invdepth_out, int check_finite, int* status, void* stream)
{
    if (levels < 1 || levels > SF_MAX_LEVELS || !grids || !s0 || !s1 || !(dt > 0.0f)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    for (int h = levels - 2; h >= -1; --h) {
        if (h == -1 && levels > 1) break;
        const int lvl = h >= 0 ? h : 0;
        ReconArgs a;
        std::memset(&a, 0, sizeof(a));
        a.H = grids[lvl].H;
        a.W = grids[lvl].W;
        a.s0 = (float4*)s0[lvl];
        a.s1 = (const float4*)s1[lvl];
        if (h >= 0) {
            a.Hc = grids[h + 1].H;
            a.Wc = grids[h + 1].W;
            a.s0c = (const float4*)s0[h + 1];
        }
        if (lvl == 0) {
            a.flow_out = flow_out;
            a.invdepth_out = invdepth_out;
            a.inv_dt = 1.0f / dt;
            a.check_finite = check_finite;
            a.status = status;
        }
        int r = launch_reconstruct(a, st);
        if (r) return r;
    }
    return SF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// allocation-free propagation (sf_propagate_noalloc)
//
// Callers that cannot allocate device memory -- code running in a stream
// callback (where CUDA calls are not allowed at all), real-time loops that
// must not touch the allocator (cudaMalloc and cudaFree can block and
// synchronise the device), or hosts whose memory pools are owned by another
// framework --
// get sf_propagate's result without cudaMalloc/cudaMallocAsync/cudaFree: the
// intermediate fields and the launch descriptors live in one file-scope
// device array that every GPU using this library holds until exit.
// ---------------------------------------------------------------------------

namespace {
constexpr size_t kNoAllocMaxPixels = size_t(1) << 20;                      // H * W per call
constexpr size_t kNoAllocDescBytes = size_t(1) << 20;                      // job + tile list
constexpr size_t kNoAllocFieldBytes = 2 * kNoAllocMaxPixels * sizeof(float4);  // (s0, s1) between launches
constexpr size_t kNoAllocJobBytes = 256;                                   // job slot ahead of the tiles
constexpr int kNoAllocMaxDevices = 64;
// the job slot must hold a PropJob and keep the int4 tile list behind it aligned
static_assert(sizeof(PropJob) <= kNoAllocJobBytes, "PropJob outgrew its slot in the allocation-free array");
static_assert(kNoAllocJobBytes % alignof(int4) == 0, "tile list behind the job slot must be int4-aligned");
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocDescBytes + kNoAllocFieldBytes];

namespace {

unsigned char* g_noalloc_addr[kNoAllocMaxDevices];   // device address of the array, per device
std::mutex g_noalloc_mutex;

// Device address of g_noalloc_scratch on the current device; looked up once
// per device (the host-side name is only a stand-in, not a device address).
int noalloc_scratch(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SF_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SF_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SF_ECUDA;
        g_noalloc_addr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_addr[dev];
    return SF_OK;
}

__global__ void k_noalloc_store_job(PropJob j, PropJob* dst) { *dst = j; }

__global__ void k_noalloc_fill_tiles(int4* work, int tiles_x, int ntiles, int T, int TH)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        work[t] = make_int4(0, (t / tiles_x) * TH, (t % tiles_x) * T, 0);
}

}  // namespace

extern "C" int sf_propagate_noalloc(const sf_grid* g, int N, int flags, float wscale, const float* s0_in,
                                    const float* s1_in, float* s0_out, float* s1_out, int* status, void* stream)
{
    if (!g || g->H < 1 || g->W < 1 || N < 1 || !s0_in || !s0_out) return SF_EINVAL;
    if ((s1_in == nullptr) != (s1_out == nullptr)) return SF_EINVAL;
    if (!aligned16(s0_in) || !aligned16(s0_out) || !aligned16(s1_in) || !aligned16(s1_out)) return SF_EINVAL;
    const size_t n = (size_t)g->H * g->W;
    if (n > kNoAllocMaxPixels) return SF_EINVAL;                 // larger frames: use sf_propagate
    const int nseg = ceil_div(N, kNfLimit);
    for (int k = 0; k < nseg; ++k) {                             // every tile list must fit
        const int nfk = N / nseg + (k < N % nseg ? 1 : 0);
        const size_t tiles = (size_t)ceil_div(g->H, prop_tile_h(nfk, prop_warps(nfk))) * ceil_div(g->W, prop_tile(nfk));
        if (kNoAllocJobBytes + tiles * sizeof(int4) > kNoAllocDescBytes) return SF_EINVAL;
    }
    unsigned char* base = nullptr;
    int r = noalloc_scratch(&base);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const bool c8 = s1_in != nullptr;
    PropJob* djob = (PropJob*)base;
    int4* dwork = (int4*)(base + kNoAllocJobBytes);
    float4* t0 = (float4*)(base + kNoAllocDescBytes);
    float4* t1 = t0 + kNoAllocMaxPixels;
    const float4* in0 = (const float4*)s0_in;
    const float4* in1 = (const float4*)s1_in;
    for (int k = 0; k < nseg && !r; ++k) {
        // the last launch writes the outputs; earlier ones alternate with the
        // scratch fields so that this holds (as in sf_propagate)
        const bool to_out = ((nseg - 1 - k) % 2) == 0;
        float4* o0 = to_out ? (float4*)s0_out : t0;
        float4* o1 = c8 ? (to_out ? (float4*)s1_out : t1) : nullptr;
        PropJob j;
        std::memset(&j, 0, sizeof(j));
        j.g = make_grid(*g);
        j.in0[0] = j.in0[1] = in0;
        j.in1[0] = j.in1[1] = in1;
        j.out0 = o0;
        j.out1 = o1;
        j.nf = N / nseg + (k < N % nseg ? 1 : 0);
        j.apply_wscale = k == 0;
        j.dt = 1.0f / (float)N;
        const int T = prop_tile(j.nf), warps = prop_warps(j.nf), TH = prop_tile_h(j.nf, warps);
        j.tiles_x = ceil_div(g->W, T);
        const int ntiles = j.tiles_x * ceil_div(g->H, TH);
        // descriptors are written by the device in stream order: the previous
        // launch has finished reading them when these kernels run
        k_noalloc_store_job<<<1, 1, 0, st>>>(j, djob);
        k_noalloc_fill_tiles<<<std::min(ceil_div(ntiles, 256), 1024), 256, 0, st>>>(dwork, j.tiles_x, ntiles, T, TH);
        r = last_error();
        if (r) break;
        Plan pl;
        pl.c8 = c8;
        pl.nf = j.nf;
        pl.warps = warps;
        pl.smem = prop_smem_bytes(warps);
        pl.jobs = djob;
        pl.work = dwork;
        pl.nwork = ntiles;
        // an ordinary launch: k_propagate reads its job and work item before
        // griddepcontrol.wait, so a programmatic launch could read the
        // descriptors before the two kernels above have written them
        r = launch_propagate(pl, 0, wscale, flags, status, st, 1.0f, /*pdl=*/false);
        in0 = o0;
        in1 = o1;
    }
    return r;
}
