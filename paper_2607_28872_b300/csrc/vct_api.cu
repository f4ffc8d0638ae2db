// C ABI of the VCT + SPH(2) library: context set-up, step orchestration,
// neighbour export and the SPH(2) derivative entry point.  Every stage of the
// path is one of the kernels in vct_kernels.cu; this file only allocates,
// launches and reads the device status word.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <optional>
#include <vector>

#include "vct_internal.cuh"

using namespace vct;

struct vct_ctx {
    DevParams P;
    cudaStream_t st;
    int64_t cap;
    int device;
    Part A, B;
    bool cur_is_A;
    Work W;
    int coop_blocks;
    int coop_blocks_mg;
    int precond;
    MG mg;
    // device mirror of a caller state for vct_step_host
    vct_state mirror;
    int64_t *row_int;          // CSR rows when the caller passes none
    double *theta_out;         // bathymetry-parameter adjoint (5 + 4 VCT_MAX_GAUSS)
    int32_t *host_status;      // pinned copy of status + stats
    int64_t last_particle;
    std::vector<void *> allocs;
    // profiling
    bool prof;
    // batched ensembles (vct_batch_step): this scenario's own stream and event,
    // and (first context of a batch) the device copy of the batch's solve jobs
    cudaStream_t bst;
    cudaEvent_t bev;
    bool rows_list;            // a batch runs this scenario's solve in the large-system form
    FlyJob *jobs_dev;
    int jobs_cap;
    unsigned char *plan_dev;   // (first context) the batched stages' job and block tables
    size_t plan_cap;
    // (first context of a batch) two side-by-side batch steps captured as a CUDA
    // graph, the batch it was captured for, and each scenario's launches in it
    cudaGraphExec_t bgraph;
    std::vector<long long> bgraph_key;
    std::vector<int64_t> bgraph_launches;
    bool bgraph_off;           // a capture failed: direct launches from then on
    cudaStream_t gst;          // the batched solve's stream
    long long serial;          // unique per context, never reused
    int graph_steps;           // steps of the current call replayed from the graph
    int64_t ppe_n;             // particles of the last pressure system still held (0: none)
    // vct_step: one step captured as a CUDA graph per state-buffer parity (the
    // sorted buffers alternate every step), replayed on a stream of its own
    cudaStream_t sst;
    cudaEvent_t sev0, sev1;
    cudaGraphExec_t sgraph[2];
    int64_t sgraph_n[2];
    int64_t sgraph_launches[2];
    bool sgraph_off;           // a capture failed: direct launches from then on
    std::vector<cudaEvent_t> ev;      // 2 per stage per profiled step
    std::vector<int> ev_stage;        // stage of each recorded pair
    int ev_used;
    double stage_ms[VCT_NSTAGES];
    int64_t stage_n[VCT_NSTAGES];
    int64_t launches;
};

namespace {

constexpr int PROF_STEPS = 512;

// Bracket a stage with events when profiling is on.
struct StageTimer {
    vct_ctx *c;
    int stage;
    int slot;
    cudaStream_t st;
    StageTimer(vct_ctx *c_, int s, cudaStream_t on = nullptr) : c(c_), stage(s), slot(-1),
        st(on ? on : c_->st)
    {
        if (c->prof && c->ev_used + 2 <= (int)c->ev.size()) {
            slot = c->ev_used;
            c->ev_used += 2;
            c->ev_stage[slot / 2] = stage;
            cudaEventRecord(c->ev[slot], st);
        }
    }
    ~StageTimer()
    {
        if (slot >= 0) cudaEventRecord(c->ev[slot + 1], st);
    }
};

void collect_times(vct_ctx *c)
{
    for (int k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]) == cudaSuccess) {
            c->stage_ms[c->ev_stage[k / 2]] += ms;
            c->stage_n[c->ev_stage[k / 2]] += 1;
        }
    }
    c->ev_used = 0;
}

vct_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? VCT_OK : VCT_ERR_CUDA; }

template <typename T>
T *dalloc(vct_ctx *c, int64_t count, cudaError_t &err)
{
    void *p = nullptr;
    if (err != cudaSuccess) return nullptr;
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    err = cudaMalloc(&p, bytes);
    if (err == cudaSuccess) {
        c->allocs.push_back(p);
        cudaMemsetAsync(p, 0, bytes, c->st);
    }
    return (T *)p;
}

void alloc_part(vct_ctx *c, Part &p, cudaError_t &e)
{
    int64_t n = c->cap;
    p.x = dalloc<double>(c, n, e); p.y = dalloc<double>(c, n, e); p.z = dalloc<double>(c, n, e);
    p.u = dalloc<double>(c, n, e); p.v = dalloc<double>(c, n, e); p.w = dalloc<double>(c, n, e);
    p.p = dalloc<double>(c, n, e); p.jbar = dalloc<double>(c, n, e);
    p.type = dalloc<int32_t>(c, n, e); p.orig = dalloc<int32_t>(c, n, e);
    p.xh = dalloc<double>(c, n, e); p.yh = dalloc<double>(c, n, e); p.zh = dalloc<double>(c, n, e);
    p.J = dalloc<double>(c, n, e); p.sx = dalloc<double>(c, n, e); p.sy = dalloc<double>(c, n, e);
    p.c0 = dalloc<double>(c, n, e); p.c3 = dalloc<double>(c, n, e);
}

Part &cur(vct_ctx *c) { return c->cur_is_A ? c->A : c->B; }
Part &alt(vct_ctx *c) { return c->cur_is_A ? c->B : c->A; }

vct_status check_state(vct_ctx *c, const vct_state *s)
{
    if (!c || !s) return VCT_ERR_ARG;
    if (s->n <= 0 || s->n > c->cap) return s->n > c->cap ? VCT_ERR_CAPACITY : VCT_ERR_ARG;
    if (!s->x || !s->z || !s->u || !s->w || !s->p || !s->jbar || !s->type) return VCT_ERR_ARG;
    if (c->P.dim == 3 && (!s->y || !s->v)) return VCT_ERR_ARG;
    return VCT_OK;
}

void reset_status(vct_ctx *c)
{
    c->launches = 0;
    c->ev_used = 0;
    cudaMemsetAsync(c->W.status, 0, sizeof(int32_t) * 4, c->st);
    cudaMemsetAsync(c->W.kiters, 0, sizeof(int32_t) * 4, c->st);
    cudaMemsetAsync(c->W.kresid, 0, sizeof(double), c->st);
}

// Reads the status word (synchronises the stream once).
vct_status finish(vct_ctx *c, vct_stats *out, int nsteps)
{
    const int graph_steps = c->graph_steps;
    c->graph_steps = 0;
    cudaError_t e = cudaMemcpyAsync(c->host_status, c->W.status, sizeof(int32_t) * 4,
                                    cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->host_status + 4, c->W.kiters, sizeof(int32_t) * 4,
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->host_status + 8, c->W.kresid, sizeof(double),
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->host_status + 10, c->W.counts, 2 * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    int code = c->host_status[0];
    c->last_particle = -1;
    if (code != 0) {
        int sorted = c->host_status[1];
        if (sorted >= 0) {
            int32_t o = -1;
            cudaMemcpy(&o, cur(c).orig + sorted, sizeof(int32_t), cudaMemcpyDeviceToHost);
            c->last_particle = o;
        }
    }
    if (c->host_status[2] != 0 && code == 0) code = VCT_ERR_TIMEOUT;
    if (out) {
        out->steps_done = code == 0 ? nsteps : 0;
        out->krylov_iters_total = c->host_status[4];
        out->krylov_iters_max = c->host_status[5];
        double r;
        memcpy(&r, c->host_status + 8, sizeof(double));
        out->last_residual = r;
        int64_t cnt[2];
        memcpy(cnt, c->host_status + 10, sizeof cnt);
        out->ppe_rows = cnt[0];
        out->ppe_nnz = cnt[1];
        out->kernel_launches = c->launches;
        out->graph_steps = graph_steps;
        out->solve_form = c->precond ? (c->mg.fly && !c->rows_list ? 1 : 2) : 0;
        out->mg_cycle = out->solve_form == 2 ? (c->mg.rowcell ? 2 : 1) : 0;
    }
    if (c->prof) collect_times(c);
    return (vct_status)code;
}

// Map, cell sort and neighbour lists of the current positions.
void geometry(vct_ctx *c, int64_t n)
{
    c->ppe_n = 0;   // a new cell order: the held pressure system no longer matches it
    { StageTimer t(c, VCT_STAGE_MAP); launch_map_key(c->P, cur(c), c->W, n, c->st); }
    { StageTimer t(c, VCT_STAGE_SORT); launch_sort(c->P, cur(c), alt(c), c->W, n, c->st); }
    c->cur_is_A = !c->cur_is_A;
    { StageTimer t(c, VCT_STAGE_NEIGHBOURS); launch_neighbours(c->P, cur(c), c->W, n, c->st); }
    c->launches += 1 + 6 + 1;   // map_key; scan x3, scatter, cell sort, reorder; neighbours
}

// Which levels block 0 keeps in shared memory (the smallest ones, within
// budget_b bytes and at most 4096 nodes each), their offsets, and where the
// row-staging area of `stage` bytes starts.
void mg_split_shared(MG &M, long long budget_b, long long stage)
{
    const long long budget = budget_b / 4;
    long long tail = 0;
    M.first_local = M.L;
    for (int q = M.L; q >= 1; --q) {
        tail += (long long)(M.S + 4) * M.n[q];
        if (tail > budget || M.n[q] > 4096) break;
        M.first_local = q;
    }
    long long so = 0;
    for (int q = M.first_local; q <= M.L; ++q) {
        M.soff[q] = so;
        so += (long long)(M.S + 4) * M.n[q];
    }
    M.sh_floats = so;
    M.stage_off = (so * 4 + 15) / 16 * 16;
    M.smem_bytes = M.stage_off + stage;
}

// One time step on the context's stream, in three parts: everything up to the
// pressure solve, the solve, and everything after it.
void step_pre(vct_ctx *c, int64_t n, const vct_probe *pr = nullptr)
{
    geometry(c, n);
    if (c->P.kind == VCT_MAP_SIGMA && c->P.volume_mode == 2) {
        StageTimer t(c, VCT_STAGE_SMOOTHING);
        launch_smoothing(c->P, cur(c), c->W, n, c->st);
        c->launches += 1;
    }
    cudaMemsetAsync(c->W.counts, 0, 2 * sizeof(int64_t), c->st);
    if (c->P.slip) {
        launch_wall_velocity(c->P, cur(c), c->W, n, c->st);
        c->launches += 1;
    }
    { StageTimer t(c, VCT_STAGE_PASS1); launch_pass1(c->P, cur(c), c->W, n, c->st); }
    if (pr && pr->fs_in) {
        launch_force_fs(cur(c), c->W, n, pr->fs_in, c->st);
        c->launches += 1;
    }
    { StageTimer t(c, VCT_STAGE_PASS2); launch_pass2(c->P, cur(c), c->W, n, 1, c->st); }
    { StageTimer t(c, VCT_STAGE_RHS); launch_rhs(c->P, cur(c), c->W, n, c->st); }
    c->launches += 3;   // pass1, pass2, rhs
    if (c->precond) {
        StageTimer t(c, VCT_STAGE_PRECOND);
        const bool rows = !c->mg.fly || c->rows_list;
        launch_mg_setup(c->P, c->W, c->mg, n, c->st, rows);
        c->launches += mg_setup_launches(c->mg) + (rows ? 5 : 0);   // + row list: flags, scan x3, scatter
    }
}

int step_solve(vct_ctx *c, int64_t n, int step)
{
    StageTimer t(c, VCT_STAGE_KRYLOV);
    c->launches += 1;
    c->ppe_n = n;
    if (c->precond) return launch_krylov_mg(c->P, c->W, c->mg, n, c->coop_blocks_mg, c->st);
    return launch_krylov(c->P, cur(c), c->W, n, step, c->coop_blocks, c->st);
}

void step_post(vct_ctx *c, int64_t n, int step, int nsteps, const vct_probe *pr)
{
    if (pr && step == nsteps - 1) {
        launch_probe_out(c->P, cur(c), c->W, n, *pr, c->st);
        c->launches += 1;
        if (pr->x_test && pr->ppe_Ax) {
            launch_probe_ax(c->P, cur(c), c->W, n, pr->x_test, pr->ppe_Ax, c->st);
            c->launches += 2;
        }
    }
    { StageTimer t(c, VCT_STAGE_CORRECTOR); launch_corrector(c->P, cur(c), c->W, n, c->st); }
    c->launches += 1;
    if (regularise_on(c->P)) {
        StageTimer t(c, VCT_STAGE_REGULARISE);
        c->launches += launch_regularise(c->P, cur(c), c->W, n, c->st);
    }
}

// Queue one time step of the current state on the context's stream.
vct_status queue_step(vct_ctx *c, int64_t n, int step, int nsteps, const vct_probe *pr)
{
    step_pre(c, n, pr && step == nsteps - 1 ? pr : nullptr);
    if (step_solve(c, n, step)) return VCT_ERR_CUDA;
    step_post(c, n, step, nsteps, pr);
    return VCT_OK;
}

// Capture one step from buffer parity par (0: A current) on the context's step
// stream; on failure the context launches directly from then on.
void capture_step(vct_ctx *c, int64_t n, int par)
{
    cudaError_t ce = cudaSuccess;
    if (!c->sst) ce = cudaStreamCreateWithFlags(&c->sst, cudaStreamNonBlocking);
    if (ce == cudaSuccess && !c->sev0) ce = cudaEventCreateWithFlags(&c->sev0, cudaEventDisableTiming);
    if (ce == cudaSuccess && !c->sev1) ce = cudaEventCreateWithFlags(&c->sev1, cudaEventDisableTiming);
    if (c->sgraph[par]) cudaGraphExecDestroy(c->sgraph[par]);
    c->sgraph[par] = nullptr;
    if (ce != cudaSuccess) {
        c->sgraph_off = true;
        return;
    }
    const cudaStream_t saved = c->st;
    const bool cur0 = c->cur_is_A;
    const int64_t l0 = c->launches, pn0 = c->ppe_n;
    c->st = c->sst;
    c->cur_is_A = par == 0;   // the parity this graph starts from
    cudaGraph_t g = nullptr;
    ce = cudaStreamBeginCapture(c->sst, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
        const vct_status qs = queue_step(c, n, 0, 1, nullptr);
        ce = cudaStreamEndCapture(c->sst, &g);
        if (ce == cudaSuccess && qs != VCT_OK) ce = cudaErrorUnknown;
    }
    if (ce == cudaSuccess && g) ce = cudaGraphInstantiate(&c->sgraph[par], g, 0);
    if (g) cudaGraphDestroy(g);
    c->sgraph_launches[par] = c->launches - l0;
    c->launches = l0;   // nothing ran yet
    c->cur_is_A = cur0;
    c->ppe_n = pn0;
    c->st = saved;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        c->sgraph[par] = nullptr;
        c->sgraph_off = true;
    } else {
        c->sgraph_n[par] = n;
    }
}

vct_status run_steps(vct_ctx *c, vct_state *s, int nsteps, const vct_probe *pr, vct_stats *out)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (nsteps < 0) return VCT_ERR_ARG;
    const int64_t n = s->n;
    reset_status(c);
    { StageTimer t(c, VCT_STAGE_LOAD); launch_load(c->P, cur(c), *s, n, c->st); }
    c->launches += 1;
    // Steps from the captured graphs (not with a probe or stage profiling, nor
    // with VCT_STEP_NOGRAPH set): every step's work is the same but for the
    // buffer parity, so one graph per parity serves all steps of this and
    // later calls with the same particle count.  They run on the context's step
    // stream, after the load and before the store on the context's stream.
    const bool graphs = !pr && !c->prof && !c->sgraph_off && nsteps > 0 && !getenv("VCT_STEP_NOGRAPH");
    int step0 = 0;
    if (graphs) {
        for (int par = 0; par < 2 && !c->sgraph_off; ++par)
            if (!c->sgraph[par] || c->sgraph_n[par] != n) capture_step(c, n, par);
    }
    if (graphs && !c->sgraph_off) {
        cudaEventRecord(c->sev0, c->st);
        cudaStreamWaitEvent(c->sst, c->sev0, 0);
        cudaError_t e = cudaSuccess;
        for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
            const int par = c->cur_is_A ? 0 : 1;
            e = cudaGraphLaunch(c->sgraph[par], c->sst);
            c->cur_is_A = !c->cur_is_A;
            c->launches += c->sgraph_launches[par];
        }
        c->ppe_n = n;
        cudaEventRecord(c->sev1, c->sst);
        cudaStreamWaitEvent(c->st, c->sev1, 0);
        if (e != cudaSuccess) return VCT_ERR_CUDA;
        step0 = nsteps;
        c->graph_steps = nsteps;
    }
    for (int step = step0; step < nsteps; ++step) {
        v = queue_step(c, n, step, nsteps, pr);
        if (v) return v;
    }
    { StageTimer t(c, VCT_STAGE_STORE); launch_store(c->P, cur(c), *s, n, c->W.status, c->st); }
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, out, nsteps);
}

// One launch of a batched ensemble stage: the stage, its coarsening level
// (BS_MG_COARSEN), its blocks in total, the offset of its block-start table,
// whether it reads the buffers this step's reorder wrote, and the profiling
// stage it counts toward.
struct BatchLaunch {
    int stage, level, total, post_sort, group;
    size_t bs_off;
};

int batch_group(int s)
{
    switch (s) {
    case BS_ZERO: case BS_MAP_KEY: return VCT_STAGE_MAP;
    case BS_CSCAN_BLOCKS: case BS_CSCAN_TOPS: case BS_CSCAN_ADD: case BS_SCATTER: case BS_CELL_SORT:
    case BS_REORDER: return VCT_STAGE_SORT;
    case BS_NEIGHBOURS: return VCT_STAGE_NEIGHBOURS;
    case BS_SMOOTHING: case BS_JBAR_COPY: return VCT_STAGE_SMOOTHING;
    case BS_WALL_VELOCITY: case BS_PASS1: return VCT_STAGE_PASS1;
    case BS_PASS2: case BS_PASS2_ISPH: return VCT_STAGE_PASS2;
    case BS_RHS: return VCT_STAGE_RHS;
    case BS_CORRECTOR: case BS_CORRECTOR_SUM: return VCT_STAGE_CORRECTOR;
    case BS_REG_GEOM: case BS_REG_DS: case BS_REG_APPLY: return VCT_STAGE_REGULARISE;
    default: return VCT_STAGE_PRECOND;
    }
}

// Ensemble step with the scenarios side by side: every stage of the step runs
// as one launch over all scenarios (each on the blocks of its own launch of
// the stage, reading its own parameters and buffers), and one cooperative
// launch solves all pressure systems at once, each on its own share of the
// grid (blocks in proportion to its particles): about 30 launches a step
// whatever the number of scenarios.  Eligible when every scenario uses the
// multigrid solver with the same dimension and precision, and the grid holds a
// block per scenario; otherwise returns VCT_ERR_ARG (the caller then queues
// the scenarios one after another).  To the solver the batch is one system:
// when it exceeds the small-system size in total, or any scenario is a large
// system, every scenario's solve runs in the large-system form (vectors,
// staged rows, L1 gathers, 16 KB of shared levels; VCT_BATCH_FORM=fly|explicit
// overrides where it can).  Every stage runs the same device code as the
// scenario's own launch of it (compiled into a different kernel, so multiply-add
// fusion may differ: agreement to rounding); the solves' partial sums are
// grouped by the scenario's share of blocks, so results agree with vct_step to
// the solver tolerance, not bit for bit.
vct_status batch_concurrent(vct_ctx *const *ctxs, vct_state *const *states, int n_scen, int nsteps,
                            vct_stats *out)
{
    if (n_scen < 2 || getenv("VCT_BATCH_SERIAL")) return VCT_ERR_ARG;
    const int prec = ctxs[0]->P.precision, dim = ctxs[0]->P.dim;
    double wsum = 0.0;
    bool any_expl = false;
    for (int k = 0; k < n_scen; ++k) {
        const vct_ctx *c = ctxs[k];
        if (!c->precond || c->P.precision != prec || c->P.dim != dim) return VCT_ERR_ARG;
        any_expl |= !c->mg.fly;
        wsum += (double)states[k]->n;
    }
    bool expl = any_expl || !krylov_mg_fly_default((long long)wsum, dim);
    if (const char *bf = getenv("VCT_BATCH_FORM")) {
        if (!strcmp(bf, "fly") && !any_expl) expl = false;
        if (!strcmp(bf, "explicit")) expl = true;
    }
    // each job's multigrid descriptor: the context's, its shared levels re-split
    // for the large-system form when the batch uses that form
    std::vector<MG> mgs(n_scen);
    size_t smem = 0;
    const long long stage = expl ? (long long)krylov_batch_stage_bytes(prec, dim) : 0;
    for (int k = 0; k < n_scen; ++k) {
        mgs[k] = ctxs[k]->mg;
        if (expl && ctxs[k]->mg.fly) {
            MG &M = mgs[k];
            M.fly = 0;
            M.staged = 1;
            M.gather_l1 = 1;
            long long budget_b = 16 * 1024;
            if (budget_b > 110 * 1024 - stage) budget_b = 110 * 1024 - stage;
            mg_split_shared(M, budget_b, stage);
        }
        if ((size_t)mgs[k].smem_bytes > smem) smem = (size_t)mgs[k].smem_bytes;
    }
    const int total = krylov_fly_batch_blocks(prec, dim, smem, expl);
    if (total < n_scen) return VCT_ERR_ARG;
    // blocks per scenario: in proportion to its particles, at least one, at most
    // one group of G lanes per row
    const int G = dim == 2 ? 4 : 8;
    std::vector<int> nb(n_scen);
    int used = 0;
    for (int k = 0; k < n_scen; ++k) {
        long long want = ((long long)states[k]->n * G + 255) / 256;
        int b = (int)((double)total * (double)states[k]->n / wsum);
        if (b < 1) b = 1;
        if (b > want) b = (int)want;
        if (b > 4096) b = 4096;
        nb[k] = b;
        used += b;
    }
    while (used > total) {   // trim the largest shares until the grid fits
        int kmax = 0;
        for (int k = 1; k < n_scen; ++k)
            if (nb[k] > nb[kmax]) kmax = k;
        if (nb[kmax] <= 1) return VCT_ERR_ARG;
        --nb[kmax];
        --used;
    }
    std::vector<FlyJob> jobs(n_scen);
    unsigned b0 = 0;
    for (int k = 0; k < n_scen; ++k) {
        const vct_ctx *c = ctxs[k];
        FlyJob &j = jobs[k];
        j.W = c->W;
        j.M = mgs[k];
        j.n = (int)states[k]->n;
        j.maxit = c->P.max_iter;
        j.rtol = c->P.rtol;
        j.inner_floor = c->P.inner_floor;
        j.b0 = b0;
        j.nb = (unsigned)nb[k];
        b0 += (unsigned)nb[k];
    }
    // The batched stages of one step, in step order: every stage some scenario
    // runs, with its block-start table (each scenario's blocks are those of its
    // own launch of the stage).  Stages up to the reorder read the state buffers
    // current at the step's start, the rest the other set.
    std::vector<BatchLaunch> plan;
    std::vector<int> tables;
    bool too_big = false;
    auto add = [&](int s, int level) {
        BatchLaunch L;
        L.stage = s;
        L.level = level;
        L.post_sort = s >= BS_NEIGHBOURS;
        L.group = batch_group(s);
        L.bs_off = tables.size();
        int64_t total = 0;
        tables.push_back(0);
        for (int k = 0; k < n_scen; ++k) {
            const vct_ctx *c = ctxs[k];
            const bool rows = !c->mg.fly || expl;
            total += batch_stage_blocks(s, c->P, c->W, mgs[k], states[k]->n, rows, level);
            if (total > (int64_t)INT32_MAX / 2) too_big = true;
            tables.push_back((int)(too_big ? 0 : total));
        }
        L.total = (int)(too_big ? 0 : total);
        if (L.total > 0) plan.push_back(L);
        else tables.resize(L.bs_off);
    };
    for (int s = BS_ZERO; s <= BS_MG_LEVEL1; ++s) add(s, 0);
    int maxl = 0;
    for (int k = 0; k < n_scen; ++k) {
        const int l = batch_coarsen_levels(mgs[k]);
        if (l > maxl) maxl = l;
    }
    for (int l = 1; l < maxl; ++l) add(BS_MG_COARSEN, l);
    add(BS_MG_COARSEN_SMALL, 0);
    const size_t n_pre = plan.size();   // the pressure solve runs after these
    for (int s = BS_CORRECTOR; s <= BS_REG_APPLY; ++s) add(s, 0);
    if (too_big) return VCT_ERR_ARG;
    // device copy: the job table of each buffer parity, then the block tables
    const size_t sj_bytes = sizeof(StageJob) * (size_t)n_scen;
    const size_t plan_bytes = 2 * sj_bytes + sizeof(int) * tables.size();
    std::vector<unsigned char> hplan(plan_bytes);
    for (int k = 0; k < n_scen; ++k) {
        vct_ctx *c = ctxs[k];
        for (int t = 0; t < 2; ++t) {
            StageJob j;
            memset(&j, 0, sizeof j);
            j.n = states[k]->n;
            j.cur = t == 0 ? cur(c) : alt(c);
            j.alt = t == 0 ? alt(c) : cur(c);
            j.W = c->W;
            j.P = c->P;
            j.M = mgs[k];
            memcpy(hplan.data() + (size_t)t * sj_bytes + sizeof(StageJob) * (size_t)k, &j, sizeof j);
        }
    }
    memcpy(hplan.data() + 2 * sj_bytes, tables.data(), sizeof(int) * tables.size());
    vct_ctx *c0 = ctxs[0];
    cudaStream_t main = c0->st;   // the caller's: job table upload
    cudaError_t e = cudaSuccess;
    if (c0->jobs_cap < n_scen) {
        if (c0->jobs_dev) cudaFree(c0->jobs_dev);
        c0->jobs_dev = nullptr;
        c0->jobs_cap = 0;
        e = cudaMalloc((void **)&c0->jobs_dev, sizeof(FlyJob) * (size_t)n_scen);
        if (e != cudaSuccess) return VCT_ERR_CUDA;
        c0->jobs_cap = n_scen;
    }
    if (c0->plan_cap < plan_bytes) {
        if (c0->plan_dev) cudaFree(c0->plan_dev);
        c0->plan_dev = nullptr;
        c0->plan_cap = 0;
        e = cudaMalloc((void **)&c0->plan_dev, plan_bytes);
        if (e != cudaSuccess) return VCT_ERR_CUDA;
        c0->plan_cap = plan_bytes;
    }
    e = cudaMemcpyAsync(c0->jobs_dev, jobs.data(), sizeof(FlyJob) * (size_t)n_scen,
                        cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c0->plan_dev, hplan.data(), plan_bytes, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(main);   // jobs and hplan are host temporaries
    for (int k = 0; k < n_scen && e == cudaSuccess; ++k) {
        vct_ctx *c = ctxs[k];
        if (!c->bst) e = cudaStreamCreateWithFlags(&c->bst, cudaStreamNonBlocking);
        if (e == cudaSuccess && !c->bev) e = cudaEventCreateWithFlags(&c->bev, cudaEventDisableTiming);
    }
    // the batched steps run on a stream of the first context's own (a graph
    // cannot be captured on the legacy default stream a caller may pass)
    if (e == cudaSuccess && !c0->gst) e = cudaStreamCreateWithFlags(&c0->gst, cudaStreamNonBlocking);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    main = c0->gst;
    const StageJob *T[2] = {reinterpret_cast<const StageJob *>(c0->plan_dev),
                            reinterpret_cast<const StageJob *>(c0->plan_dev + sj_bytes)};
    const int *tb = reinterpret_cast<const int *>(c0->plan_dev + 2 * sj_bytes);
    std::vector<cudaStream_t> saved(n_scen);
    bool prof = false;
    for (int k = 0; k < n_scen; ++k) {
        vct_ctx *c = ctxs[k];
        saved[k] = c->st;
        c->st = c->bst;
        c->rows_list = expl;
        prof |= c->prof;
        reset_status(c);
        launch_load(c->P, cur(c), *states[k], states[k]->n, c->st);
        c->launches += 1;
        cudaEventRecord(c->bev, c->st);   // the steps start after every scenario's load
        cudaStreamWaitEvent(main, c->bev, 0);
    }
    // One step on the batch stream: the batched stages up to the solve, the
    // batched solve, the batched stages after it.  Step `step` of the call
    // starts from job table step % 2 (each scenario's buffers alternate every
    // step).  The launches are counted on the first context; with profiling on,
    // its stage times are the batch's.
    auto one_step = [&](int step) -> cudaError_t {
        const StageJob *X = T[step & 1], *Y = T[(step + 1) & 1];
        std::optional<StageTimer> t;   // brackets a run of launches of one profiling stage
        int grp = -1;
        auto run = [&](const BatchLaunch &L) {
            if (prof && L.group != grp) {
                t.reset();
                t.emplace(c0, L.group, main);
                grp = L.group;
            }
            launch_batched(L.stage, dim, prec, L.post_sort ? Y : X, tb + L.bs_off, n_scen, L.total,
                           L.level, main);
            c0->launches += 1;
        };
        for (size_t q = 0; q < n_pre; ++q) run(plan[q]);
        t.reset();
        grp = -1;
        int le;
        {
            StageTimer tk(c0, VCT_STAGE_KRYLOV, main);
            le = launch_krylov_fly_batch(prec, dim, c0->jobs_dev, n_scen, b0, smem, expl, main);
        }
        c0->launches += 1;
        for (size_t q = n_pre; q < plan.size(); ++q) run(plan[q]);
        t.reset();
        for (int k = 0; k < n_scen; ++k) {
            ctxs[k]->cur_is_A = !ctxs[k]->cur_is_A;
            ctxs[k]->ppe_n = states[k]->n;
        }
        return le ? (cudaError_t)le : cudaSuccess;
    };
    // Steps in pairs from a CUDA graph: the state buffers alternate every step,
    // so after two steps every pointer is back where it started and one captured
    // pair serves all pairs of this and later calls with the same batch.  Not
    // with stage profiling (its events are per step), nor with VCT_BATCH_NOGRAPH
    // set; if a capture fails, direct launches from then on.
    int step0 = 0;
    if (nsteps >= 2 && !prof && !c0->bgraph_off && !getenv("VCT_BATCH_NOGRAPH")) {
        std::vector<long long> key = {n_scen, expl ? 1 : 0, (long long)smem, (long long)b0,
                                      (long long)(intptr_t)c0->jobs_dev,
                                      (long long)(intptr_t)c0->plan_dev, (long long)plan_bytes};
        for (int k = 0; k < n_scen; ++k) {
            key.push_back(ctxs[k]->serial);
            key.push_back(states[k]->n);
            key.push_back(ctxs[k]->cur_is_A ? 1 : 0);
        }
        if (!c0->bgraph || key != c0->bgraph_key) {
            if (c0->bgraph) cudaGraphExecDestroy(c0->bgraph);
            c0->bgraph = nullptr;
            c0->bgraph_key.clear();
            const int64_t l0 = c0->launches;
            std::vector<char> cur0(n_scen);
            std::vector<int64_t> pn0(n_scen);
            for (int k = 0; k < n_scen; ++k) {
                cur0[k] = ctxs[k]->cur_is_A;
                pn0[k] = ctxs[k]->ppe_n;
            }
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed);
            cudaError_t se = cudaSuccess;
            if (ce == cudaSuccess) {
                for (int q = 0; q < 2 && se == cudaSuccess; ++q) se = one_step(q);
                ce = cudaStreamEndCapture(main, &g);
            }
            if (ce == cudaSuccess && se == cudaSuccess && g)
                ce = cudaGraphInstantiate(&c0->bgraph, g, 0);
            else if (ce == cudaSuccess)
                ce = se;
            if (g) cudaGraphDestroy(g);
            c0->bgraph_launches.assign(1, c0->launches - l0);
            c0->launches = l0;   // nothing ran yet
            for (int k = 0; k < n_scen; ++k) {
                ctxs[k]->cur_is_A = cur0[k] != 0;
                ctxs[k]->ppe_n = pn0[k];
            }
            if (ce != cudaSuccess) {
                cudaGetLastError();   // the failed capture launched nothing
                c0->bgraph = nullptr;
                c0->bgraph_off = true;
            } else {
                c0->bgraph_key = key;
            }
        }
        if (c0->bgraph) {
            const int pairs = nsteps / 2;
            for (int q = 0; q < pairs && e == cudaSuccess; ++q) e = cudaGraphLaunch(c0->bgraph, main);
            c0->launches += (int64_t)pairs * c0->bgraph_launches[0];
            for (int k = 0; k < n_scen; ++k) {
                ctxs[k]->graph_steps = 2 * pairs;
                ctxs[k]->ppe_n = states[k]->n;
            }
            step0 = 2 * pairs;
        }
    }
    for (int step = step0; step < nsteps && e == cudaSuccess; ++step) e = one_step(step);
    cudaEventRecord(c0->bev, main);   // the stores after the last step
    for (int k = 0; k < n_scen; ++k) {
        vct_ctx *c = ctxs[k];
        cudaStreamWaitEvent(c->st, c0->bev, 0);
        launch_store(c->P, cur(c), *states[k], states[k]->n, c->W.status, c->st);
        c->launches += 1;
    }
    vct_status first = e == cudaSuccess ? VCT_OK : VCT_ERR_CUDA;
    if (!first && cudaGetLastError() != cudaSuccess) first = VCT_ERR_CUDA;
    for (int k = 0; k < n_scen; ++k) {
        vct_status v = finish(ctxs[k], out ? out + k : nullptr, nsteps);
        if (!first) first = v;
        ctxs[k]->st = saved[k];
        ctxs[k]->rows_list = false;
    }
    return first;
}

}  // namespace

extern "C" {
#define VCT_API __attribute__((visibility("default")))

VCT_API vct_status vct_init(vct_ctx **out, const vct_bathymetry *bathy, vct_map_kind kind,
                    double aspect_ratio, const vct_params *prm, int64_t capacity, void *stream)
{
    if (!out || !bathy || !prm) return VCT_ERR_ARG;
    *out = nullptr;
    if (prm->dim != 2 && prm->dim != 3) return VCT_ERR_ARG;
    if ((int)kind < 0 || (int)kind > 3) return VCT_ERR_ARG;
    if (!(prm->d0 > 0) || !(prm->dt > 0) || !(prm->rho > 0) || capacity <= 0 ||
        capacity > (int64_t)INT32_MAX / 4)
        return VCT_ERR_ARG;
    if (bathy->n_gauss < 0 || bathy->n_gauss > VCT_MAX_GAUSS) return VCT_ERR_ARG;
    if (!(prm->ops_shift >= 0.0) || !(prm->ds_overlap >= 0.0 && prm->ds_overlap < 1.0) ||
        !(prm->xsph_eps >= 0.0))
        return VCT_ERR_ARG;
    if (bathy->n_gauss > 0 && (!bathy->amp || !bathy->cx || !bathy->cy || !bathy->width))
        return VCT_ERR_ARG;
    if ((kind == VCT_MAP_E || kind == VCT_MAP_BFE) && !(aspect_ratio > 0)) return VCT_ERR_ARG;
    if (kind == VCT_MAP_SIGMA && !(prm->H_hat > 0 && prm->alpha_min > 0 &&
                                   prm->alpha_max >= prm->alpha_min))
        return VCT_ERR_ARG;
    if (prm->precision != VCT_FP64 && prm->precision != VCT_MIXED) return VCT_ERR_ARG;
    if (prm->volume_mode < 0 || prm->volume_mode > 2) return VCT_ERR_ARG;
    if (prm->spin_limit < 0) return VCT_ERR_ARG;
    if (prm->operators != 0 && prm->operators != 1) return VCT_ERR_ARG;
    if (prm->wall_slip != 0 && prm->wall_slip != 1) return VCT_ERR_ARG;
    if (!(prm->cell_over_re == 0.0 || prm->cell_over_re >= 1.0) || !(prm->mg_omega >= 0.0) ||
        !(prm->mg_kappa >= 0.0) || prm->solve_form < 0 || prm->solve_form > 2 ||
        prm->mg_cycle < 0 || prm->mg_cycle > 2)
        return VCT_ERR_ARG;
    // the background cell grid, validated before anything is allocated
    int grid_nc[3];
    int64_t ncell = 1;
    {
        vct_status gs = cell_grid(prm, (prm->cell_over_re > 0.0 ? prm->cell_over_re : 1.0) *
                                           prm->re_over_l * (prm->l_over_d0 * prm->d0),
                                  (int64_t)INT32_MAX / 2, grid_nc, &ncell);
        if (gs != VCT_OK) return gs;
    }

    static long long serials = 0;
    vct_ctx *c = new (std::nothrow) vct_ctx();
    if (!c) return VCT_ERR_ARG;
    c->serial = __atomic_add_fetch(&serials, 1, __ATOMIC_RELAXED);
    c->st = (cudaStream_t)stream;
    c->cap = capacity;
    cudaGetDevice(&c->device);
    DevParams &P = c->P;
    memset(&P, 0, sizeof P);
    P.dim = prm->dim;
    P.kind = (int)kind;
    P.smag = prm->smagorinsky;
    P.volume_mode = prm->volume_mode;
    P.n_gauss = bathy->n_gauss;
    P.max_nbr = prm->max_neighbours > 0 ? prm->max_neighbours : (prm->dim == 2 ? 64 : 160);
    P.precision = prm->precision;
    P.max_iter = prm->krylov_max_iter > 0 ? prm->krylov_max_iter : 1000;
    P.aspect = aspect_ratio;
    P.rho = prm->rho;
    P.nu_k = prm->nu_k;
    P.g = prm->g;
    P.dt = prm->dt;
    P.d0 = prm->d0;
    // l, r_e and r_e^2 formed exactly as the parameters define them
    P.l = prm->l_over_d0 * prm->d0;
    P.inv_l = 1.0 / P.l;
    P.re = prm->re_over_l * P.l;
    P.re2 = P.re * P.re;
    P.V0 = prm->dim == 2 ? prm->d0 * prm->d0 : prm->d0 * prm->d0 * prm->d0;
    P.ad = prm->dim == 2 ? 10.0 / (7.0 * M_PI * P.l * P.l) : 1.0 / (M_PI * P.l * P.l * P.l);
    P.gamma = prm->gamma_over_dt * prm->dt;
    P.cv = prm->cv_over_dt * prm->dt;
    P.cs = prm->cs;
    P.ds = prm->ds;
    P.H = prm->H;
    P.H_hat = prm->H_hat;
    P.amin = prm->alpha_min;
    P.amax = prm->alpha_max;
    P.lam_lo = prm->lam_fs_lo;
    P.lam_hi = prm->lam_fs_hi;
    P.rtol = prm->krylov_rtol;
    P.ops_shift = prm->ops_shift;
    P.ds_overlap = prm->ds_overlap;
    P.xsph_eps = prm->xsph_eps;
    P.operators = prm->operators;
    P.slip = prm->wall_slip;
    P.pguess = getenv("VCT_PGUESS") ? atoi(getenv("VCT_PGUESS")) : 2;   // 0: none, 1: linear
    P.inner_floor = prm->precision == VCT_MIXED ? 1e-4 : 0.0;
    if (prm->precision == VCT_MIXED && getenv("VCT_INNER_FLOOR")) P.inner_floor = atof(getenv("VCT_INNER_FLOOR"));
    P.cell_h = (prm->cell_over_re > 0.0 ? prm->cell_over_re : 1.0) * P.re;
    P.inv_cell_h = 1.0 / P.cell_h;
    for (int k = 0; k < 3; ++k) {
        P.box_lo[k] = prm->box_lo[k];
        P.nc[k] = grid_nc[k];
    }
    P.h0 = bathy->h0;
    P.slope_x = bathy->slope_x;
    P.slope_y = bathy->slope_y;
    P.cos_amp = bathy->cos_amp;
    P.cos_len = bathy->cos_len;
    for (int g = 0; g < bathy->n_gauss; ++g) {
        P.gamp[g] = bathy->amp[g];
        P.gcx[g] = bathy->cx[g];
        P.gcy[g] = bathy->cy[g];
        P.gwid[g] = bathy->width[g];
        P.ginv2[g] = 1.0 / (bathy->width[g] * bathy->width[g]);
    }

    cudaError_t e = cudaSuccess;
    const int64_t n = capacity, d = prm->dim, m = d == 2 ? 3 : 6, K = P.max_nbr;
    alloc_part(c, c->A, e);
    alloc_part(c, c->B, e);
    c->cur_is_A = true;
    Work &W = c->W;
    W.cap = n;
    W.max_nbr = (int32_t)K;
    W.ncell = ncell;
    W.key = dalloc<int32_t>(c, n, e);
    W.cell_count = dalloc<int32_t>(c, ncell + 1, e);
    W.cell_start = dalloc<int32_t>(c, ncell + 1, e);
    W.cursor = dalloc<int32_t>(c, ncell, e);
    W.perm = dalloc<int32_t>(c, n, e);
    W.scan_tmp = dalloc<int32_t>(c, (ncell > n ? ncell : n) + 1024, e);
    W.row_tmp = dalloc<int64_t>(c, n / 1024 + 1024, e);
    W.nbr_cnt = dalloc<int32_t>(c, n, e);
    W.nbr = dalloc<int32_t>(c, n * K, e);
    W.L = dalloc<double>(c, n * d * d, e);
    W.gv = dalloc<double>(c, n * d * d, e);
    W.Ct = dalloc<double>(c, n * d * m, e);
    W.rho_hat = dalloc<double>(c, n, e);
    W.lam = dalloc<double>(c, n, e);
    W.nu = dalloc<double>(c, n, e);
    W.fs = dalloc<int32_t>(c, n, e);
    W.vstar = dalloc<double>(c, n * d, e);
    W.acc = dalloc<double>(c, n * d, e);
    W.pcnt = dalloc<int32_t>(c, n, e);
    const int64_t Kb = (K + 7) / 8 * 8;   // whole slot blocks (ell_at)
    W.pcol = dalloc<int32_t>(c, n * Kb, e);
    W.pval = dalloc<double>(c, prm->precision == VCT_MIXED ? 1 : n * Kb, e);
    W.pvalf = dalloc<float>(c, prm->precision == VCT_MIXED ? n * Kb : 1, e);
    W.diag = dalloc<double>(c, n, e);
    W.bvec = dalloc<double>(c, n, e);
    W.wallrhs = dalloc<double>(c, n, e);
    W.pwall = dalloc<double>(c, n * d, e);
    W.jbar_tmp = dalloc<double>(c, n, e);
    W.jratio = dalloc<double>(c, n, e);
    W.hatf = dalloc<float4>(c, n, e);
    W.hatlo = dalloc<float4>(c, n, e);
    W.velhi = dalloc<float4>(c, n, e);
    W.vello = dalloc<float4>(c, n, e);
    W.vshi = dalloc<float4>(c, n, e);
    W.vslo = dalloc<float4>(c, n, e);
    W.vol = dalloc<double>(c, n, e);
    W.volf = dalloc<float>(c, n, e);
    W.adj = dalloc<double>(c, n * 3 * (m + d), e);   // the operator adjoint's rows, up to 3 fields at once
    if (prm->ops_shift > 0.0 || prm->ds_overlap > 0.0 || prm->xsph_eps > 0.0) {
        W.rxh = dalloc<double>(c, n * d, e);
        W.rmet = dalloc<double>(c, n * 3, e);
        W.rud = dalloc<double>(c, n * d, e);
        W.rdh = dalloc<double>(c, n * d, e);
    }
    W.kx = dalloc<double>(c, n, e);
    W.urow_flag = dalloc<int32_t>(c, n, e);
    W.urow_pos = dalloc<int32_t>(c, n + 1, e);
    W.urow = dalloc<int32_t>(c, n, e);
    W.p_last = dalloc<double>(c, n, e);
    W.p_prev = dalloc<double>(c, n, e);
    W.p_prev2 = dalloc<double>(c, n, e);
    if (e == cudaSuccess) {   // NaN: no history yet
        cudaMemset(W.p_last, 0xFF, sizeof(double) * (size_t)n);
        cudaMemset(W.p_prev, 0xFF, sizeof(double) * (size_t)n);
        cudaMemset(W.p_prev2, 0xFF, sizeof(double) * (size_t)n);
    }
    W.kr = dalloc<double>(c, n, e);
    W.krh = dalloc<double>(c, n, e);
    W.kp0 = dalloc<double>(c, n, e);
    W.kp1 = dalloc<double>(c, n, e);
    W.kv0 = dalloc<double>(c, n, e);
    W.kv1 = dalloc<double>(c, n, e);
    W.kt = dalloc<double>(c, n, e);
    W.ks = dalloc<double>(c, n, e);
    W.kd = dalloc<double>(c, n, e);
    W.kf = dalloc<double>(c, n, e);
    c->coop_blocks = krylov_coop_blocks(prm->precision, prm->dim);
    c->precond = prm->preconditioner == 1;
    {   // multigrid hierarchy over the cell grid
        MG &M = c->mg;
        memset(&M, 0, sizeof M);
        M.S = prm->dim == 2 ? 9 : 27;
        // tuned: 2-D wave (42k particles, 100 steps, kappa 1.3), iterations per step
        // by omega: 0.7 17.4, 0.75 16.5, 0.8 15.8, 0.85 15.2, 0.9 15.0 (kappa 1.1-1.4
        // within 1.5 of these); with the hierarchy down to 64 nodes: 0.8 15.6,
        // 0.85 15.2, 0.9 14.9 (in 3-D, 0.8 already diverges); with the coarse levels'
        // own damping (below) 0.85 is as fast as 0.9; 3-D BFE
        // beach (aspect 4, 2.1M particles), iterations per step by kappa at omega 0.7:
        // 1.8: 77, 1.5: 47, 1.4: 40, 1.3: 33, 1.2: 31 (540k slice: 1.0 36, 1.1 32,
        // 1.2 32); omega 0.8 does not converge there, 0.75 is within 1 iteration
        M.omega = prm->dim == 2 ? 0.85f : 0.7f;
        M.kappa = prm->dim == 2 ? 1.3f : 1.2f;
        M.coarse_sweeps = 24;
        M.dims[1][0] = P.nc[0];
        M.dims[1][1] = P.nc[1];
        M.dims[1][2] = P.nc[2];
        M.n[1] = (int)ncell;
        // Anisotropy of the projected operator: c_trans weights d2/dz^2 by about
        // alpha^2 (E/BFE: the aspect ratio squared; sigma: mean over the box;
        // BF: 1).  While the z coupling exceeds 2.5 x the horizontal one, coarsen
        // along z only (each such step divides the ratio by 4), then in all axes.
        double ratio = 1.0;
        if (kind == VCT_MAP_E || kind == VCT_MAP_BFE) ratio = aspect_ratio * aspect_ratio;
        else if (kind == VCT_MAP_SIGMA) {
            double acc = 0.0;
            int cnt = 0;
            for (int ix = 0; ix <= 64; ++ix)
                for (int iy = 0; iy <= (prm->dim == 3 ? 16 : 0); ++iy) {
                    double x = prm->box_lo[0] + (prm->box_hi[0] - prm->box_lo[0]) * ix / 64.0;
                    double y = prm->dim == 3 ? prm->box_lo[1] + (prm->box_hi[1] - prm->box_lo[1]) * iy / 16.0 : 0.0;
                    double h = bathy->h0 + bathy->slope_x * x + bathy->slope_y * y;
                    if (bathy->cos_amp != 0.0) h += bathy->cos_amp * cos(2.0 * M_PI * x / bathy->cos_len);
                    for (int g = 0; g < bathy->n_gauss; ++g) {
                        double dx = x - bathy->cx[g], dy = y - bathy->cy[g], w = bathy->width[g];
                        h += bathy->amp[g] * exp(-(dx * dx + dy * dy) / (2.0 * w * w));
                    }
                    double D = prm->H - h, al = D > 0 ? prm->H_hat / D : prm->alpha_max;
                    al = al < prm->alpha_min ? prm->alpha_min : (al > prm->alpha_max ? prm->alpha_max : al);
                    acc += al * al;
                    ++cnt;
                }
            ratio = acc / cnt;
        }
        int l = 1;
        // coarsen while a level has more than 64 nodes in 2-D, 4 in 3-D (with no
        // sweeps on the coarsest level; iterations and solve time per step by this
        // size, 2-D wave: 4: 15.63, 2330 us; 16: 15.52, 2275; 64: 15.37, 2205;
        // 256: 17.27, 2415; 3-D slice: 4: 31.2, 47.4 ms; 16: 31.2, 47.4; 64: 32.3, 48.7)
        const double zratio = getenv("VCT_MG_ZRATIO") ? atof(getenv("VCT_MG_ZRATIO")) : 2.5;
        const int coarsest = getenv("VCT_MG_MINN") ? atoi(getenv("VCT_MG_MINN"))
                                                   : (prm->dim == 2 ? 64 : 4);
        while (M.n[l] > coarsest && l < MG_MAXL) {
            const int agg = getenv("VCT_MG_SHIFT") ? atoi(getenv("VCT_MG_SHIFT")) : 1;
            int sh[3] = {agg, prm->dim == 3 ? agg : 0, agg};
            if (ratio > zratio && M.dims[l][2] > 1) {
                sh[0] = 0;
                sh[1] = 0;
                ratio *= 0.25;
            }
            int nx = (M.dims[l][0] + (1 << sh[0]) - 1) >> sh[0];
            int ny = (M.dims[l][1] + (1 << sh[1]) - 1) >> sh[1];
            int nz = (M.dims[l][2] + (1 << sh[2]) - 1) >> sh[2];
            if ((long long)nx * ny * nz == M.n[l]) break;
            for (int q = 0; q < 3; ++q) M.shift[l][q] = sh[q];
            M.dims[l + 1][0] = nx;
            M.dims[l + 1][1] = ny;
            M.dims[l + 1][2] = nz;
            M.n[l + 1] = nx * ny * nz;
            ++l;
        }
        M.L = l;
        // block 0 keeps the smallest levels in shared memory (<= 96 KB, <= 4096 nodes
        // per level); the rest run grid-wide.  Large systems also stage rows in
        // shared memory (every block), and the levels give way so that two solver
        // blocks still fit on an SM (<= 110 KB each).
        // VCT_MG_FORM=fly|explicit overrides the size rule (tests cover both forms)
        M.fly = krylov_mg_fly_default(n, prm->dim) ? 1 : 0;
        if (prm->solve_form) M.fly = prm->solve_form == 1 ? 1 : 0;
        if (const char *fm = getenv("VCT_MG_FORM")) {
            if (!strcmp(fm, "fly")) M.fly = 1;
            if (!strcmp(fm, "explicit")) M.fly = 0;
        }
        // large-system form (measured on the 2.1M-particle 3-D beach): staged rows,
        // L1-cached gathers and a 16 KB level budget (a small shared-memory
        // carve-out leaves L1 to the gathers) -- 5.8 vs 7.4 ms per iteration
        M.staged = M.fly ? 0 : 1;
        if (getenv("VCT_MG_STAGE")) M.staged = M.fly ? 0 : atoi(getenv("VCT_MG_STAGE"));
        M.gather_l1 = M.fly ? 0 : 1;
        if (getenv("VCT_GATHER_L1")) M.gather_l1 = atoi(getenv("VCT_GATHER_L1"));
        const long long stage = (long long)krylov_mg_stage_bytes(prm->precision, prm->dim, M.staged != 0);
        long long budget_b = M.fly ? 96 * 1024 : 16 * 1024;
        if (budget_b > 110 * 1024 - stage) budget_b = 110 * 1024 - stage;
        if (getenv("VCT_MG_SMEM_KB")) budget_b = (long long)atoi(getenv("VCT_MG_SMEM_KB")) * 1024;
        mg_split_shared(M, budget_b, stage);
        // the coarsest level has at most a few nodes: Jacobi sweeps there do not
        // pay (2-D wave, per step: 8 sweeps 15.72 iterations / 2372 us, 2 sweeps
        // 15.68 / 2310, none 15.63 / 2285)
        M.coarse_sweeps = 0;
        // large-system form (also when a batch runs a small scenario in it):
        // V(0,1) cycles through the row-cell operator by default.  Measured on
        // the 2.1M-particle 3-D beach (krylov ms per step, iterations): V(1,1)
        // 128.0 / 31.8, V(0,1) 114.1 / 47.3 (each iteration 1.9x cheaper); 64 2-D
        // scenarios side by side: 29.4 vs 46.6 ms per step.
        M.rowcell = prm->mg_cycle == 1 ? 0 : 1;
        if (getenv("VCT_MG_ROWCELL")) M.rowcell = atoi(getenv("VCT_MG_ROWCELL")) != 0;
        // the 3-D V(0,1) cycle's damping and scale (beach, krylov ms per step at
        // omega / kappa: 0.7 / 1.2 82.9, 0.8 / 1.1 80.5, 0.9 / 1.1 81.7, 0.8 / 1.0
        // 86.8, 0.8 / 0.9 106.5; the V(1,1) cycle diverges at omega 0.8)
        if (prm->dim == 3 && M.rowcell && !M.fly) {
            M.omega = 0.8f;
            M.kappa = 1.1f;
        }
        if (prm->mg_omega > 0.0) M.omega = (float)prm->mg_omega;
        if (prm->mg_kappa > 0.0) M.kappa = (float)prm->mg_kappa;
        if (getenv("VCT_MG_OMEGA")) M.omega = (float)atof(getenv("VCT_MG_OMEGA"));
        if (getenv("VCT_MG_KAPPA")) M.kappa = (float)atof(getenv("VCT_MG_KAPPA"));
        M.kappa_c = M.kappa;
        // damping on the coarse levels (measured, iterations / solve time per step):
        // 2-D wave 0.7 16.35 / 2.28 ms, 0.8 15.35 / 2.15, 0.9 (= fine) 14.89 / 2.08,
        // 1.0 14.60 / 2.05, 1.1 14.32 / 2.01, and with the fine damping 0.85 and
        // 1.0 here 14.35 / 2.01 (the default: no over-relaxation anywhere); 3-D
        // slice 0.6 32.3 / 48.6 ms, 0.7 (= fine) 31.2 / 46.9, 0.8 30.1 / 45.3,
        // 0.85 30.5 / 46.2, 0.9 30.5 / 45.9
        M.omega_c = prm->dim == 2 ? 1.0f : 0.8f;
        if (getenv("VCT_MG_OMEGA_C")) M.omega_c = (float)atof(getenv("VCT_MG_OMEGA_C"));
        if (getenv("VCT_MG_KAPPA_C")) M.kappa_c = (float)atof(getenv("VCT_MG_KAPPA_C"));
        if (getenv("VCT_MG_SWEEPS")) M.coarse_sweeps = atoi(getenv("VCT_MG_SWEEPS"));
        M.presmooth = 1;
        if (getenv("VCT_MG_PRESMOOTH")) M.presmooth = atoi(getenv("VCT_MG_PRESMOOTH"));
        long long pos = 0;
        for (int q = 1; q <= M.L; ++q) {
            M.offA[q] = pos;
            pos += (long long)M.S * M.n[q];
            M.offv[q] = pos;
            pos += 4LL * M.n[q];
        }
        W.mg_pool = dalloc<float>(c, pos, e);
        W.mg_dsc = dalloc<float>(c, n, e);
        W.mg_B = M.rowcell ? dalloc<float>(c, (int64_t)M.S * n, e) : nullptr;
        W.cellid = dalloc<int32_t>(c, n, e);
        W.kr0 = dalloc<double>(c, n, e);
        W.kq0 = dalloc<double>(c, n, e);
        W.kq1 = dalloc<double>(c, n, e);
        W.kz0 = dalloc<double>(c, n, e);
        W.kzb = dalloc<double>(c, n, e);
        c->coop_blocks_mg = krylov_mg_coop_blocks(prm->precision, prm->dim, (size_t)M.smem_bytes, M.fly != 0);
        if (getenv("VCT_SOLVE_BLOCKS")) {   // cap on the solve's grid (tuning)
            const int cap_b = atoi(getenv("VCT_SOLVE_BLOCKS"));
            if (cap_b > 0 && cap_b < c->coop_blocks_mg) c->coop_blocks_mg = cap_b;
        }
    }
    if (c->coop_blocks <= 0) e = e == cudaSuccess ? cudaErrorInvalidConfiguration : e;
    W.partial = dalloc<double>(c, (int64_t)8 * 4096, e);   // k-major, 4096 blocks max
    W.scal = dalloc<double>(c, 16, e);
    W.kiters = dalloc<int32_t>(c, 4, e);
    W.kresid = dalloc<double>(c, 1, e);
    W.bar = dalloc<unsigned int>(c, 2, e);
    W.spin_limit = prm->spin_limit > 0 ? (unsigned long long)prm->spin_limit : SPIN_LIMIT_DEFAULT;
    W.status = dalloc<int32_t>(c, 4, e);
    W.counts = dalloc<long long>(c, 2, e);
    c->row_int = dalloc<int64_t>(c, n + 1, e);
    c->theta_out = dalloc<double>(c, 5 + 4 * VCT_MAX_GAUSS, e);
    c->mirror.x = dalloc<double>(c, n, e);
    c->mirror.y = dalloc<double>(c, n, e);
    c->mirror.z = dalloc<double>(c, n, e);
    c->mirror.u = dalloc<double>(c, n, e);
    c->mirror.v = dalloc<double>(c, n, e);
    c->mirror.w = dalloc<double>(c, n, e);
    c->mirror.p = dalloc<double>(c, n, e);
    c->mirror.jbar = dalloc<double>(c, n, e);
    c->mirror.type = dalloc<int32_t>(c, n, e);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->host_status, 64);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        vct_destroy(c);
        return VCT_ERR_CUDA;
    }
    c->last_particle = -1;
    *out = c;
    return VCT_OK;
}

VCT_API vct_status vct_set_stream(vct_ctx *c, void *stream)
{
    if (!c) return VCT_ERR_ARG;
    c->st = (cudaStream_t)stream;
    return VCT_OK;
}

VCT_API vct_status vct_reset_history(vct_ctx *c)
{
    if (!c) return VCT_ERR_ARG;
    const size_t bytes = sizeof(double) * (size_t)c->cap;
    cudaError_t e = cudaMemsetAsync(c->W.p_last, 0xFF, bytes, c->st);   // NaN: no history
    if (e == cudaSuccess) e = cudaMemsetAsync(c->W.p_prev, 0xFF, bytes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->W.p_prev2, 0xFF, bytes, c->st);
    return e == cudaSuccess ? VCT_OK : VCT_ERR_CUDA;
}

VCT_API vct_status vct_build_neighbours(vct_ctx *c, const vct_state *s, int64_t *row_ptr, int32_t *col,
                                int64_t col_cap, int64_t *nnz)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    int64_t *rows = row_ptr ? row_ptr : c->row_int;
    launch_csr_export(c->P, cur(c), c->W, n, rows, nullptr, 0, c->st);
    int64_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, rows + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    if (nnz) *nnz = total;
    if (col) {
        if (total > col_cap) return VCT_ERR_CAPACITY;
        launch_csr_export(c->P, cur(c), c->W, n, rows, col, col_cap, c->st);
    }
    return finish(c, nullptr, 0);
}

VCT_API vct_status sph2_derivatives(vct_ctx *c, const vct_state *s, const double *phi, int32_t ncomp,
                            double *grad_hat, double *d2_hat, double *lap_phys)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!phi || ncomp <= 0) return VCT_ERR_ARG;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_pass1(c->P, cur(c), c->W, n, c->st);
    launch_sph2_field(c->P, cur(c), c->W, n, phi, ncomp, grad_hat, d2_hat, lap_phys, c->st);
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

VCT_API vct_status sph2_derivatives_backward(vct_ctx *c, const vct_state *s, int32_t ncomp,
                                             const double *grad_hat_bar, const double *d2_hat_bar,
                                             const double *lap_phys_bar, double *phi_bar)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!phi_bar || ncomp <= 0) return VCT_ERR_ARG;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_pass1(c->P, cur(c), c->W, n, c->st);
    launch_sph2_adjoint(c->P, cur(c), c->W, n, ncomp, grad_hat_bar, d2_hat_bar, lap_phys_bar,
                        phi_bar, c->st);
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

VCT_API vct_status sph2_gradient_backward_positions(vct_ctx *c, const vct_state *s,
                                                    const double *phi, int32_t ncomp,
                                                    const double *grad_hat_bar, double *xh_bar)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!phi || !grad_hat_bar || !xh_bar || ncomp <= 0 || ncomp > 3) return VCT_ERR_ARG;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_gradpos(c->P, cur(c), c->W, n, ncomp, phi, grad_hat_bar, xh_bar, c->st);
    c->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

// The second-derivative position adjoints keep per-particle factors and
// adjoints (30 doubles in 2-D, 72 in 3-D) in the pressure coefficients' storage,
// roundup(max_neighbours, 4 / 8) slots per particle of doubles (FP64 form) or
// floats (mixed form).
static bool d2pos_scratch_fits(const vct_ctx *c)
{
    const int64_t eg = c->P.dim == 2 ? 4 : 8, need = c->P.dim == 2 ? 30 : 72;
    const int64_t kb = ((int64_t)c->W.max_nbr + eg - 1) / eg * eg;
    return (c->P.precision == VCT_MIXED ? kb / 2 : kb) >= need;
}

VCT_API vct_status sph2_d2_backward_positions(vct_ctx *c, const vct_state *s, const double *phi,
                                              const double *d2_hat_bar, double *xh_bar)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!phi || !d2_hat_bar || !xh_bar) return VCT_ERR_ARG;
    if (!d2pos_scratch_fits(c)) return VCT_ERR_CAPACITY;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_d2pos(c->P, cur(c), c->W, n, false, phi, d2_hat_bar, xh_bar, c->st);
    c->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

VCT_API vct_status vct_ppe_backward_positions(vct_ctx *c, const vct_state *s, const double *x,
                                              const double *p_bar, double *xh_bar)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!x || !p_bar || !xh_bar) return VCT_ERR_ARG;
    if (!d2pos_scratch_fits(c)) return VCT_ERR_CAPACITY;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_pass1(c->P, cur(c), c->W, n, c->st);   // free-surface flags: the unknown rows
    launch_d2pos(c->P, cur(c), c->W, n, true, x, p_bar, xh_bar, c->st);
    c->launches += 4;
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

VCT_API vct_status vct_rho_backward_positions(vct_ctx *c, const vct_state *s,
                                              const double *rho_bar, double *xh_bar)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!rho_bar || !xh_bar) return VCT_ERR_ARG;
    const int64_t n = s->n;
    reset_status(c);
    launch_load(c->P, cur(c), *s, n, c->st);
    geometry(c, n);
    launch_rhopos(c->P, cur(c), c->W, n, rho_bar, xh_bar, c->st);
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return finish(c, nullptr, 0);
}

VCT_API vct_status vct_map_backward(vct_ctx *c, const vct_state *s, const double *zh_bar,
                                    const double *J_bar, const double *sx_bar,
                                    const double *sy_bar, const double *c0_bar,
                                    const double *c3_bar, double *theta_bar)
{
    if (!c || !s || !theta_bar) return VCT_ERR_ARG;
    if (s->n <= 0 || s->n > c->cap) return s->n > c->cap ? VCT_ERR_CAPACITY : VCT_ERR_ARG;
    if (!s->x || !s->z || (c->P.dim == 3 && !s->y)) return VCT_ERR_ARG;
    const int nparam = 5 + 4 * c->P.n_gauss;
    // device table of the six adjoint pointers lives in the context's scratch
    const double *tab[6] = {zh_bar, J_bar, sx_bar, sy_bar, c0_bar, c3_bar};
    cudaError_t e = cudaMemcpyAsync(c->W.scal, tab, sizeof tab, cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    double *out = c->theta_out;   // 5 + 4 * VCT_MAX_GAUSS doubles
    if (launch_map_adjoint(c->P, *s, s->n, (const double *const *)c->W.scal, c->W.adj,
                           c->cap * (c->P.dim == 2 ? 5 : 9), out, c->st))
        return VCT_ERR_CAPACITY;
    e = cudaMemcpyAsync(theta_bar, out, sizeof(double) * nparam, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return VCT_OK;
}

VCT_API vct_status vct_map_backward_positions(vct_ctx *c, const vct_state *s, const double *zh_bar,
                                              const double *J_bar, const double *sx_bar,
                                              const double *sy_bar, const double *c0_bar,
                                              const double *c3_bar, double *pos_bar)
{
    if (!c || !s || !pos_bar) return VCT_ERR_ARG;
    if (s->n <= 0 || s->n > c->cap) return s->n > c->cap ? VCT_ERR_CAPACITY : VCT_ERR_ARG;
    if (!s->x || !s->z || (c->P.dim == 3 && !s->y)) return VCT_ERR_ARG;
    const double *tab[6] = {zh_bar, J_bar, sx_bar, sy_bar, c0_bar, c3_bar};
    cudaError_t e = cudaMemcpyAsync(c->W.scal, tab, sizeof tab, cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    launch_map_pos_adjoint(c->P, *s, s->n, (const double *const *)c->W.scal, pos_bar, c->st);
    e = cudaStreamSynchronize(c->st);   // tab is a host temporary
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    return VCT_OK;
}

VCT_API vct_status vct_gauge_loss(vct_ctx *c, const vct_state *s, const int32_t *fs, int32_t n_gauges,
                                  const double *gauges, double *loss, double *eta, double *pos_bar)
{
    if (!c || !s || !fs || !gauges || !loss) return VCT_ERR_ARG;
    if (s->n <= 0 || s->n > c->cap) return s->n > c->cap ? VCT_ERR_CAPACITY : VCT_ERR_ARG;
    if (!s->x || !s->z || !s->type || (c->P.dim == 3 && !s->y)) return VCT_ERR_ARG;
    if (n_gauges < 1 || n_gauges > 16) return VCT_ERR_ARG;
    // gauge positions (x, y; y = 0 in 2-D) and the results in the context's small scratch
    double gxy[32];
    for (int g = 0; g < n_gauges; ++g) {
        gxy[2 * g] = gauges[(c->P.dim == 3 ? 2 : 1) * g];
        gxy[2 * g + 1] = c->P.dim == 3 ? gauges[2 * g + 1] : 0.0;
        if (!(gxy[2 * g] > -1.0e300 && gxy[2 * g] < 1.0e300) ||
            !(gxy[2 * g + 1] > -1.0e300 && gxy[2 * g + 1] < 1.0e300))
            return VCT_ERR_ARG;
    }
    double *gdev = c->theta_out, *res = c->theta_out + 32;
    cudaError_t e = cudaMemcpyAsync(gdev, gxy, sizeof(double) * 2 * n_gauges, cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    const int rc = launch_gauge_loss(c->P, *s, s->n, fs, n_gauges, gdev, c->W.adj,
                                     c->cap * (c->P.dim == 2 ? 5 : 9), res, pos_bar, c->st);
    if (rc) return VCT_ERR_CAPACITY;
    double out[3 * 16 + 1];
    e = cudaMemcpyAsync(out, res, sizeof(double) * (3 * n_gauges + 1), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    *loss = out[3 * n_gauges];
    if (eta)
        for (int g = 0; g < n_gauges; ++g) eta[g] = out[2 * n_gauges + g];
    return VCT_OK;
}

VCT_API vct_status vct_step(vct_ctx *c, vct_state *s, int32_t nsteps, vct_stats *out)
{
    return run_steps(c, s, nsteps, nullptr, out);
}

VCT_API vct_status vct_batch_step(vct_ctx *const *ctxs, vct_state *const *states, int32_t n_scen,
                                  int32_t nsteps, vct_stats *out)
{
    if (!ctxs || !states || n_scen <= 0 || nsteps < 0) return VCT_ERR_ARG;
    for (int k = 0; k < n_scen; ++k) {
        vct_status v = check_state(ctxs[k], states[k]);
        if (v) return v;
        for (int q = 0; q < k; ++q)
            if (ctxs[q] == ctxs[k]) return VCT_ERR_ARG;   // one context per scenario
    }
    {
        vct_status b = batch_concurrent(ctxs, states, n_scen, nsteps, out);
        if (b != VCT_ERR_ARG) return b;   // VCT_ERR_ARG: not eligible, run the serial form
    }
    // every scenario's work goes to the first context's stream, in order
    cudaStream_t st = ctxs[0]->st;
    std::vector<cudaStream_t> saved(n_scen);
    for (int k = 0; k < n_scen; ++k) {
        saved[k] = ctxs[k]->st;
        ctxs[k]->st = st;
        reset_status(ctxs[k]);
        launch_load(ctxs[k]->P, cur(ctxs[k]), *states[k], states[k]->n, st);
        ctxs[k]->launches += 1;
    }
    vct_status first = VCT_OK;
    for (int step = 0; step < nsteps && !first; ++step)
        for (int k = 0; k < n_scen && !first; ++k)
            first = queue_step(ctxs[k], states[k]->n, step, nsteps, nullptr);
    for (int k = 0; k < n_scen; ++k) {
        launch_store(ctxs[k]->P, cur(ctxs[k]), *states[k], states[k]->n, ctxs[k]->W.status, st);
        ctxs[k]->launches += 1;
    }
    if (!first && cudaGetLastError() != cudaSuccess) first = VCT_ERR_CUDA;
    for (int k = 0; k < n_scen; ++k) {
        vct_status v = finish(ctxs[k], out ? out + k : nullptr, nsteps);
        if (!first) first = v;
        ctxs[k]->st = saved[k];
    }
    return first;
}

// Transposed pressure solve on the held system, with the Jacobi-preconditioned
// BiCGSTAB as the fallback when the forward hierarchy does not carry it.
static vct_status ppe_adjoint_solve(vct_ctx *c, int64_t n, const double *p_bar, double *b_bar,
                                    vct_stats *out)
{
    vct_status v = VCT_ERR_NOCONV;
    if (c->precond) {
        // A^T in place of A, its own multigrid hierarchy and the forward solver
        // (the form the context uses for A) on it, then A restored
        reset_status(c);
        launch_ppe_transpose(c->P, c->W, n, true, c->st);
        const bool rows = !c->mg.fly || c->rows_list;
        launch_mg_setup(c->P, c->W, c->mg, n, c->st, rows);
        launch_adj_gather(cur(c), c->W, n, p_bar, c->st);
        const int e = launch_krylov_mg(c->P, c->W, c->mg, n, c->coop_blocks_mg, c->st);
        launch_adj_scatter(cur(c), c->W, n, b_bar, c->st);
        launch_ppe_transpose(c->P, c->W, n, false, c->st);
        c->launches += 2 + mg_setup_launches(c->mg) + (rows ? 5 : 0) + 1 + 1 + 1 + 1;
        if (e || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
        v = finish(c, out, 1);
    }
    if (v == VCT_ERR_NOCONV) {
        // no hierarchy, or it did not carry A^T: the Jacobi-preconditioned BiCGSTAB
        reset_status(c);
        const int e = launch_ppe_adjoint(c->P, cur(c), c->W, n, p_bar, b_bar, c->st);
        c->launches += 4;   // gather, transposed slots, solve, scatter
        if (e || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
        v = finish(c, out, 1);
    }
    return v;
}

VCT_API vct_status vct_ppe_adjoint(vct_ctx *c, const double *p_bar, double *b_bar, vct_stats *out)
{
    if (!c || !p_bar || !b_bar) return VCT_ERR_ARG;
    if (c->ppe_n <= 0) return VCT_ERR_ARG;   // no pressure system held
    return ppe_adjoint_solve(c, c->ppe_n, p_bar, b_bar, out);
}

VCT_API vct_status vct_step_backward_velocity(vct_ctx *c, const vct_state *s, const double *v_bar,
                                              const double *x_bar, const double *p_bar,
                                              double *v_bar_in, vct_stats *out)
{
    vct_status v = check_state(c, s);
    if (v) return v;
    if (!v_bar_in) return VCT_ERR_ARG;
    const int64_t n = s->n;
    const int d = c->P.dim;
    const bool reg = regularise_on(c->P);
    if (!c->W.sadj) {
        cudaError_t e = cudaSuccess;
        c->W.sadj = dalloc<double>(c, c->cap * (4 * d + 2 * d * d + 1), e);
        c->W.sadj_co = dalloc<double>(c, c->cap * (3 * d + d * d + 2), e);
        if (e != cudaSuccess) {
            c->W.sadj = c->W.sadj_co = nullptr;
            return VCT_ERR_CUDA;
        }
    }
    if (reg && !c->W.radj) {
        cudaError_t e = cudaSuccess;
        // + the step-start positions, velocities and FP32 position copies kept
        //   across the forward run (6 doubles and 2 float4 per particle)
        c->W.radj = dalloc<double>(c, c->cap * (regadj_rows(d) + 2 * d + 10), e);
        if (e != cudaSuccess) {
            c->W.radj = nullptr;
            return VCT_ERR_CUDA;
        }
    }
    bool assembled = false;
    if (reg) {
        // The regularisation acts last, on the corrector's x' and u': run the
        // step forward up to it, take its reverse first (into u'_bar, x'_bar),
        // then the rest of the step's reverse from there, on the operators this
        // forward run assembled (the positions, velocities and FP32 position
        // copies that the corrector and the regularisation overwrite are kept
        // and put back).
        double *vb_co = c->W.radj + (int64_t)regadj_rows(d) * c->cap, *xb_co = vb_co + d * n;
        reset_status(c);
        launch_load(c->P, cur(c), *s, n, c->st);
        c->launches += 1;
        step_pre(c, n);
        const Part pc = cur(c);
        double *keep = c->W.radj + (int64_t)(regadj_rows(d) + 2 * d) * c->cap;
        double *fields[6] = {pc.x, pc.y, pc.z, pc.u, pc.v, pc.w};
        const size_t nb8 = sizeof(double) * (size_t)n, nb16 = sizeof(float4) * (size_t)n;
        cudaError_t ce = cudaSuccess;
        for (int q = 0; q < 6 && ce == cudaSuccess; ++q)
            ce = cudaMemcpyAsync(keep + q * c->cap, fields[q], nb8, cudaMemcpyDeviceToDevice, c->st);
        float4 *keepf = reinterpret_cast<float4 *>(keep + 6 * c->cap);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(keepf, c->W.hatf, nb16, cudaMemcpyDeviceToDevice, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(keepf + c->cap, c->W.hatlo, nb16, cudaMemcpyDeviceToDevice, c->st);
        if (ce != cudaSuccess) return VCT_ERR_CUDA;
        if (step_solve(c, n, 0)) return VCT_ERR_CUDA;
        launch_corrector(c->P, cur(c), c->W, n, c->st);
        launch_regadj_save(c->P, cur(c), c->W, n, c->st);
        c->launches += 2 + launch_regularise(c->P, cur(c), c->W, n, c->st);
        launch_regadj(c->P, cur(c), c->W, n, v_bar, x_bar, vb_co, xb_co, c->st);
        c->launches += 4;
        for (int q = 0; q < 6 && ce == cudaSuccess; ++q)
            ce = cudaMemcpyAsync(fields[q], keep + q * c->cap, nb8, cudaMemcpyDeviceToDevice, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(c->W.hatf, keepf, nb16, cudaMemcpyDeviceToDevice, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(c->W.hatlo, keepf + c->cap, nb16, cudaMemcpyDeviceToDevice, c->st);
        if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
        v = finish(c, nullptr, 0);
        if (v) return v;
        // the corrector wrote the pressure history of the context: clear it
        if (vct_reset_history(c) != VCT_OK) return VCT_ERR_CUDA;
        v_bar = vb_co;
        x_bar = xb_co;
        assembled = true;
    }
    reset_status(c);
    if (!assembled) {
        launch_load(c->P, cur(c), *s, n, c->st);
        c->launches += 1;
        step_pre(c, n);   // the step's operators at the given positions (no solve, no update)
    }
    launch_stepadj_a(c->P, cur(c), c->W, n, v_bar, x_bar, p_bar, c->st);
    c->launches += 2 + (c->P.smag ? 2 : 0);
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    v = finish(c, nullptr, 0);   // errors of the operators' assembly
    if (v) return v;
    c->ppe_n = n;
    double *pb = c->W.sadj_co, *bb = c->W.sadj_co + n, *lb = c->W.sadj_co + 2 * n;
    v = ppe_adjoint_solve(c, n, pb, bb, out);
    if (v) return v;
    reset_status(c);
    // the transposed solve kept its slot table in the neighbour lists: list the
    // neighbours again (the same lists: same sorted positions)
    launch_neighbours(c->P, cur(c), c->W, n, c->st);
    c->launches += 1;
    launch_stepadj_b(c->P, cur(c), c->W, n, c->st);
    // the eddy viscosity's share reaches the velocities through the corrected
    // gradient: the SPH(2) adjoint takes it as the gradient's adjoint
    const double *gb = c->P.smag ? c->W.sadj_co + (2 + 3 * d) * n : nullptr;
    if (c->P.operators == 1) launch_isph_adjoint(c->P, cur(c), c->W, n, d, gb, lb, v_bar_in, c->st);
    else launch_sph2_adjoint(c->P, cur(c), c->W, n, d, gb, nullptr, lb, v_bar_in, c->st);
    launch_stepadj_c(c->P, cur(c), c->W, n, v_bar_in, c->st);
    c->launches += 2 + (c->P.smag ? 2 : 0) + 2 * d + 1 + (c->P.slip ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return VCT_ERR_CUDA;
    v = finish(c, nullptr, 0);
    if (out) out->kernel_launches = c->launches;
    return v;
}

VCT_API vct_status vct_step_probe(vct_ctx *c, vct_state *s, const vct_probe *pr, vct_stats *out)
{
    if (!pr) return VCT_ERR_ARG;
    return run_steps(c, s, 1, pr, out);
}

VCT_API vct_status vct_step_host(vct_ctx *c, vct_state *h, int32_t nsteps, vct_stats *out)
{
    if (!c || !h) return VCT_ERR_ARG;
    if (h->n <= 0 || h->n > c->cap) return h->n > c->cap ? VCT_ERR_CAPACITY : VCT_ERR_ARG;
    if (!h->x || !h->z || !h->u || !h->w || !h->p || !h->jbar || !h->type) return VCT_ERR_ARG;
    const bool d3 = c->P.dim == 3;
    if (d3 && (!h->y || !h->v)) return VCT_ERR_ARG;
    const size_t bd = sizeof(double) * (size_t)h->n;
    vct_state m = c->mirror;
    m.n = h->n;
    cudaError_t e = cudaSuccess;
    double *src[8] = {h->x, h->y, h->z, h->u, h->v, h->w, h->p, h->jbar};
    double *dst[8] = {m.x, m.y, m.z, m.u, m.v, m.w, m.p, m.jbar};
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
        if (!src[k]) continue;
        e = cudaMemcpyAsync(dst[k], src[k], bd, cudaMemcpyHostToDevice, c->st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)m.type, h->type, sizeof(int32_t) * (size_t)h->n,
                            cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    if (!d3) { m.y = nullptr; m.v = nullptr; }
    vct_status v = run_steps(c, &m, nsteps, nullptr, out);
    if (v != VCT_OK) return v;
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
        if (!src[k] || !dst[k] || (!d3 && (k == 1 || k == 4))) continue;
        e = cudaMemcpyAsync(src[k], dst[k], bd, cudaMemcpyDeviceToHost, c->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return cuda_ok(e);
}

VCT_API vct_status vct_set_profiling(vct_ctx *c, int32_t on)
{
    if (!c) return VCT_ERR_ARG;
    if (on && c->ev.empty()) {
        c->ev.resize(2 * VCT_NSTAGES * PROF_STEPS);
        c->ev_stage.resize(VCT_NSTAGES * PROF_STEPS);
        for (auto &e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return VCT_ERR_CUDA;
    }
    c->prof = on != 0;
    c->ev_used = 0;
    for (int k = 0; k < VCT_NSTAGES; ++k) {
        c->stage_ms[k] = 0.0;
        c->stage_n[k] = 0;
    }
    return VCT_OK;
}

VCT_API vct_status vct_stage_times(vct_ctx *c, double *ms, int64_t *launches)
{
    if (!c || !ms) return VCT_ERR_ARG;
    for (int k = 0; k < VCT_NSTAGES; ++k) {
        ms[k] = c->stage_ms[k];
        if (launches) launches[k] = c->stage_n[k];
    }
    return VCT_OK;
}

VCT_API vct_status vct_last_error(vct_ctx *c, int64_t *particle)
{
    if (!c || !particle) return VCT_ERR_ARG;
    *particle = c->last_particle;
    return VCT_OK;
}

VCT_API const char *vct_strerror(vct_status s)
{
    switch (s) {
    case VCT_OK: return "ok";
    case VCT_ERR_ARG: return "invalid argument";
    case VCT_ERR_CUDA: return "CUDA runtime error";
    case VCT_ERR_CAPACITY: return "capacity exceeded (particles or neighbours)";
    case VCT_ERR_SINGULAR: return "singular correction or moment matrix";
    case VCT_ERR_NONFINITE: return "non-finite state";
    case VCT_ERR_NOCONV: return "pressure solve did not converge";
    case VCT_ERR_TIMEOUT: return "device spin-wait timed out";
    }
    return "unknown status";
}

VCT_API void vct_destroy(vct_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->bst) {
        cudaStreamSynchronize(c->bst);
        cudaStreamDestroy(c->bst);
    }
    if (c->bev) cudaEventDestroy(c->bev);
    if (c->jobs_dev) cudaFree(c->jobs_dev);
    if (c->plan_dev) cudaFree(c->plan_dev);
    if (c->bgraph) cudaGraphExecDestroy(c->bgraph);
    for (int par = 0; par < 2; ++par)
        if (c->sgraph[par]) cudaGraphExecDestroy(c->sgraph[par]);
    if (c->sst) {
        cudaStreamSynchronize(c->sst);
        cudaStreamDestroy(c->sst);
    }
    if (c->sev0) cudaEventDestroy(c->sev0);
    if (c->sev1) cudaEventDestroy(c->sev1);
    if (c->gst) {
        cudaStreamSynchronize(c->gst);
        cudaStreamDestroy(c->gst);
    }
    for (auto &e : c->ev) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    if (c->host_status) cudaFreeHost(c->host_status);
    delete c;
}

}  // extern "C"
