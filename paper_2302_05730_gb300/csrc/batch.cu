// Batched m-Cubes: many independent integrations of uneven dimension and sample budget run
// together. Per iteration there is one persistent V-Sample launch per (d, integrand) class, then
// one Rebin launch over every (job, axis) pair. The whole iteration schedule is captured once
// into a CUDA graph and launched as a single graph. The autotuner times candidate launch shapes
// per dimension. The per-job arithmetic is exactly the single-job path's (vsample.cuh); a job
// draws with Philox counter word 3 = its index in the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/mcubes.h"
#include "internal.h"
#include "vsample.cuh"
#include "vsample64.cuh"

using namespace mcubes;

namespace {

constexpr int kGS = kNB + 1;

using BatchLauncher = int (*)(int, const BatchJob *, const BatchTile *, int, int, int, int, int, const LaunchReq &,
                              cudaStream_t);

BatchLauncher batch_launcher_for(int prec, int fid)
{
    static const BatchLauncher f64[10] = {
        launch_vsample_batch_f64_0, launch_vsample_batch_f64_1, launch_vsample_batch_f64_2,
        launch_vsample_batch_f64_3, launch_vsample_batch_f64_4, launch_vsample_batch_f64_5,
        launch_vsample_batch_f64_6, launch_vsample_batch_f64_7, launch_vsample_batch_f64_8,
        launch_vsample_batch_f64_9};
    static const BatchLauncher f32[10] = {
        launch_vsample_batch_f32_0, launch_vsample_batch_f32_1, launch_vsample_batch_f32_2,
        launch_vsample_batch_f32_3, launch_vsample_batch_f32_4, launch_vsample_batch_f32_5,
        launch_vsample_batch_f32_6, launch_vsample_batch_f32_7, launch_vsample_batch_f32_8,
        launch_vsample_batch_f32_9};
    return prec == MCUBES_FP32_EVAL ? f32[fid] : f64[fid];
}

__global__ void batch_uniform_grids(double *const *grids, const int *dims, int n_jobs)
{
    const int j = blockIdx.x;
    if (j >= n_jobs) return;
    double *g = grids[j];
    const int n = dims[j] * kGS;
    for (int e = threadIdx.x; e < n; e += blockDim.x) g[e] = (double)(e % kGS) / (double)kNB;
}

struct Shape {
    int threads = kMaxBlockThreads;
    int cpt = 4;
    int hist = 0;
};

Shape shape_for(const mcubes_batch_tuning *tune, int d)
{
    Shape s;
    if (tune) {
        if (tune->block_threads[d] > 0) s.threads = tune->block_threads[d];
        if (tune->cubes_per_thread[d] > 0) s.cpt = tune->cubes_per_thread[d];
        s.hist = tune->hist_mode[d];
    }
    return s;
}

bool shape_ok(const Shape &s)
{
    return s.threads >= 64 && s.threads <= kMaxBlockThreads && s.threads % 32 == 0 && s.cpt >= 1 &&
           s.cpt <= 4096 && (s.hist == 0 || s.hist == 1);
}

// Device state of one batch: jobs, grids, bin contributions, sums and the tile lists.
struct Plan {
    int n_jobs = 0, itmax = 0, prec = 0;
    std::vector<Problem> pb;
    char *dmem = nullptr;           // one allocation for everything
    BatchJob *d_jobs = nullptr;
    double *d_sums = nullptr;       // n_jobs x itmax x 2
    double *d_C = nullptr;          // all jobs' bin contributions, contiguous
    size_t C_doubles = 0;
    double **d_gridptr[2] = {nullptr, nullptr};
    double **d_Cptr = nullptr;
    int *d_dims = nullptr;
    uint32_t *d_rb_job = nullptr, *d_rb_axis = nullptr;
    int n_rebin_blocks = 0;
    // classes (d, fid) with their tiles
    struct Class {
        int d, fid;
        Shape shape;
        BatchTile *d_tiles = nullptr;
        int n_tiles = 0;
        size_t samples = 0;
    };
    std::vector<Class> classes;
    std::vector<BatchTile> h_tiles_all;   // kept for re-tiling
    std::map<std::pair<int, int>, bool> fast;   // FP64 (d, family) classes whose jobs all take the fast kernel

    ~Plan() { release(); }
    void release()
    {
        for (auto &c : classes)
            if (c.d_tiles) cudaFree(c.d_tiles);
        classes.clear();
        if (dmem) cudaFree(dmem);
        dmem = nullptr;
    }

    int init(int n, const mcubes_job *jobs, int itmax_, int iter_adjust, int precision, int plain64 = 0)
    {
        n_jobs = n;
        itmax = itmax_;
        prec = precision;
        pb.resize(n);
        for (int j = 0; j < n; ++j) {
            const mcubes_job &J = jobs[j];
            const int st = prepare(J.integrand_id, J.params, J.d, J.ncall, J.seed, 0, (uint32_t)j,
                                   iter_adjust > 0, precision, pb[j]);
            if (st) return st;
        }
        // one device allocation: jobs | sums | C | grids | pointer tables | dims | rebin tables
        size_t grid_doubles = 0, C_d = 0;
        for (const auto &p : pb) {
            grid_doubles += (size_t)p.d * kGS;
            C_d += (size_t)p.d * kNB;
            n_rebin_blocks += p.d;
        }
        C_doubles = C_d;
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t b_jobs = al(sizeof(BatchJob) * n), b_sums = al(sizeof(double) * 2 * n * (size_t)itmax);
        const size_t b_C = al(sizeof(double) * C_d), b_grid = al(sizeof(double) * grid_doubles);
        const size_t b_ptr = al(sizeof(double *) * n), b_dims = al(sizeof(int) * n);
        const size_t b_rb = al(sizeof(uint32_t) * n_rebin_blocks);
        const size_t total = b_jobs + b_sums + b_C + 2 * b_grid + 3 * b_ptr + b_dims + 2 * b_rb;
        int st = cuda_status(mc_malloc((void **)&dmem, total));
        if (st) return st;
        char *q = dmem;
        d_jobs = (BatchJob *)q; q += b_jobs;
        d_sums = (double *)q; q += b_sums;
        d_C = (double *)q; q += b_C;
        double *grid0 = (double *)q; q += b_grid;
        double *grid1 = (double *)q; q += b_grid;
        d_gridptr[0] = (double **)q; q += b_ptr;
        d_gridptr[1] = (double **)q; q += b_ptr;
        d_Cptr = (double **)q; q += b_ptr;
        d_dims = (int *)q; q += b_dims;
        d_rb_job = (uint32_t *)q; q += b_rb;
        d_rb_axis = (uint32_t *)q; q += b_rb;

        // FP64 classes of the six Genz families take the fast kernel when every job's fold is usable;
        // their jobs' parameters then carry it
        fast.clear();
        if (precision == MCUBES_FP64 && !plain64) {
            for (int j = 0; j < n; ++j) {
                const std::pair<int, int> key{pb[j].d, pb[j].fid};
                VsampleParams Q = pb[j].P;
                const bool ok = fast64_fold(pb[j].fid, Q, pb[j].d) &&
                                fast64_smem_bytes_rt(pb[j].d, pb[j].fid, 1) <= (size_t)227 * 1024;
                auto it = fast.find(key);
                fast[key] = (it == fast.end() ? true : it->second) && ok;
            }
        }
        std::vector<BatchJob> hj(n);
        std::vector<double *> g0(n), g1(n), cp(n);
        std::vector<int> dims(n);
        std::vector<uint32_t> rbj, rba;
        size_t go = 0, co = 0;
        for (int j = 0; j < n; ++j) {
            const Problem &p = pb[j];
            std::memset(&hj[j], 0, sizeof(BatchJob));
            hj[j].P = p.P;
            if (fast.count({p.d, p.fid}) && fast[{p.d, p.fid}]) fast64_fold(p.fid, hj[j].P, p.d);
            hj[j].P.probe = nullptr;
            hj[j].P.probe_mask = 0xFFFFFFFFu;
            g0[j] = grid0 + go;
            g1[j] = grid1 + go;
            cp[j] = d_C + co;
            hj[j].grid[0] = g0[j];
            hj[j].grid[1] = g1[j];
            hj[j].C = cp[j];
            hj[j].sums = d_sums + 2 * (size_t)itmax * j;
            dims[j] = p.d;
            for (int a = 0; a < p.d; ++a) {
                rbj.push_back((uint32_t)j);
                rba.push_back((uint32_t)a);
            }
            go += (size_t)p.d * kGS;
            co += (size_t)p.d * kNB;
        }
        st = cuda_status(cudaMemcpy(d_jobs, hj.data(), sizeof(BatchJob) * n, cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_gridptr[0], g0.data(), sizeof(double *) * n, cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_gridptr[1], g1.data(), sizeof(double *) * n, cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_Cptr, cp.data(), sizeof(double *) * n, cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_dims, dims.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_rb_job, rbj.data(), sizeof(uint32_t) * rbj.size(), cudaMemcpyHostToDevice));
        if (!st) st = cuda_status(cudaMemcpy(d_rb_axis, rba.data(), sizeof(uint32_t) * rba.size(), cudaMemcpyHostToDevice));
        return st;
    }

    // (Re)build the tile lists of every class for the given tuning.
    int tile(const mcubes_batch_tuning *tune)
    {
        for (auto &c : classes)
            if (c.d_tiles) cudaFree(c.d_tiles);
        classes.clear();
        std::map<std::pair<int, int>, std::vector<int>> members;
        for (int j = 0; j < n_jobs; ++j) members[{pb[j].d, pb[j].fid}].push_back(j);
        for (auto &kv : members) {
            Class c;
            c.d = kv.first.first;
            c.fid = kv.first.second;
            c.shape = shape_for(tune, c.d);
            if (!shape_ok(c.shape)) return MCUBES_ERR_INVALID_ARG;
            const auto fi = fast.find(kv.first);
            if (fi != fast.end() && fi->second) c.shape.hist = 2;   // the fast FP64 kernel (shared histogram)
            const uint64_t per = (uint64_t)c.shape.threads * (uint64_t)c.shape.cpt;
            std::vector<BatchTile> tl;
            for (int j : kv.second) {
                const uint64_t m = (uint64_t)pb[j].m;
                for (uint64_t c0 = 0; c0 < m; c0 += per) {
                    const uint64_t c1 = std::min(m, c0 + per);
                    tl.push_back(BatchTile{(uint32_t)j, (uint32_t)c0, (uint32_t)c1, 0u});
                }
                c.samples += (size_t)(m * (uint64_t)pb[j].p);
            }
            c.n_tiles = (int)tl.size();
            int st = cuda_status(mc_malloc((void **)&c.d_tiles, sizeof(BatchTile) * tl.size()));
            if (!st) st = cuda_status(cudaMemcpy(c.d_tiles, tl.data(), sizeof(BatchTile) * tl.size(), cudaMemcpyHostToDevice));
            classes.push_back(c);
            if (st) return st;
        }
        return MCUBES_OK;
    }

    int launch_class(const Class &c, int it, int parity, int adjust, cudaStream_t s) const
    {
        LaunchReq req;
        int st = make_req(nullptr, req);
        if (st) return st;
        req.threads = c.shape.threads;
        req.user_threads = 1;
        req.blocks_per_sm = 0;
        return cuda_status((cudaError_t)batch_launcher_for(prec, c.fid)(c.d, d_jobs, c.d_tiles, c.n_tiles, it, parity,
                                                                         adjust, c.shape.hist, req, s));
    }

    // Enqueue the whole schedule on s: uniform grids, zero sums, then per iteration zero C,
    // V-Sample every class, Rebin every (job, axis).
    int enqueue(int iter_adjust, cudaStream_t s) const
    {
        batch_uniform_grids<<<n_jobs, 256, 0, s>>>(d_gridptr[0], d_dims, n_jobs);
        int st = cuda_status(cudaGetLastError());
        if (!st) st = cuda_status(cudaMemsetAsync(d_sums, 0, sizeof(double) * 2 * (size_t)n_jobs * itmax, s));
        int parity = 0;
        for (int it = 0; it < itmax && !st; ++it) {
            const int adjust = it < iter_adjust;
            if (adjust) st = cuda_status(cudaMemsetAsync(d_C, 0, sizeof(double) * C_doubles, s));
            for (const auto &c : classes) {
                if (st) break;
                st = launch_class(c, it, parity, adjust, s);
            }
            if (!st && adjust && it + 1 < itmax) {
                st = cuda_status((cudaError_t)launch_rebin_batch(
                    n_rebin_blocks, d_rb_job, d_rb_axis, (const double *const *)d_gridptr[parity],
                    (const double *const *)d_Cptr, d_gridptr[1 - parity], 1.5, s));
                parity = 1 - parity;
            }
        }
        return st;
    }
};

int check_jobs(int n_jobs, const mcubes_job *jobs)
{
    if (n_jobs < 1 || !jobs) return MCUBES_ERR_INVALID_ARG;
    for (int j = 0; j < n_jobs; ++j)
        if (!jobs[j].params) return MCUBES_ERR_INVALID_ARG;
    return MCUBES_OK;
}

void combine_job(const double *sums, int itmax, double m, mcubes_result *r)
{
    std::vector<double> I(itmax), V(itmax);
    bool finite = true;
    for (int it = 0; it < itmax; ++it) {
        I[it] = sums[2 * it] / m;
        V[it] = sums[2 * it + 1] / (m * m);
        finite = finite && std::isfinite(I[it]) && std::isfinite(V[it]);
    }
    if (!finite) {
        r->status = MCUBES_ERR_NONFINITE;
        return;
    }
    int nzero = 0;
    double zsum = 0.0;
    for (int it = 0; it < itmax; ++it)
        if (V[it] == 0.0) {
            ++nzero;
            zsum += I[it];
        }
    if (nzero > 0) {
        r->estimate = zsum / nzero;
        r->error = 0.0;
        r->chi2_dof = 0.0;
    } else {
        double sw = 0.0, swI = 0.0;
        for (int it = 0; it < itmax; ++it) {
            sw += 1.0 / V[it];
            swI += I[it] / V[it];
        }
        const double Ibar = swI / sw;
        double chi = 0.0;
        for (int it = 0; it < itmax; ++it) chi += (I[it] - Ibar) * (I[it] - Ibar) / V[it];
        r->estimate = Ibar;
        r->error = 1.0 / std::sqrt(sw);
        r->chi2_dof = itmax > 1 ? chi / (double)(itmax - 1) : 0.0;
    }
    r->status = MCUBES_OK;
}

}  // namespace

extern "C" int mcubes_integrate_batch(int n_jobs, const mcubes_job *jobs, int itmax, int iter_adjust, int precision,
                                      const mcubes_batch_tuning *tune, void *stream, mcubes_result *out,
                                      double *iter_out)
{
    int st = check_jobs(n_jobs, jobs);
    if (!out) st = MCUBES_ERR_INVALID_ARG;
    if (!st && (itmax < 1 || itmax > 0xFFFF || iter_adjust < 0 || iter_adjust > itmax)) st = MCUBES_ERR_INVALID_ARG;
    if (st) return st;
    std::memset(out, 0, sizeof(mcubes_result) * n_jobs);

    if (tune && tune->fp64_plain != 0 && tune->fp64_plain != 1) return MCUBES_ERR_INVALID_ARG;

    Plan plan;
    if ((st = plan.init(n_jobs, jobs, itmax, iter_adjust, precision, tune ? tune->fp64_plain : 0))) return st;
    if ((st = plan.tile(tune))) return st;

    cudaStream_t run = nullptr;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&run, cudaStreamNonBlocking)))) return st;
    cudaStream_t user = (cudaStream_t)stream;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (run) cudaStreamDestroy(run);
    };
    if (user) {
        st = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (!st) st = cuda_status(cudaEventRecord(ev, user));
        if (!st) st = cuda_status(cudaStreamWaitEvent(run, ev, 0));
    }
    // First use of each kernel instance sets its shared-memory limit and occupancy; do that
    // outside the capture (a launch over zero tiles does only the set-up).
    for (const auto &c : plan.classes) {
        if (st) break;
        Plan::Class none = c;
        none.n_tiles = 0;
        st = plan.launch_class(none, 0, 0, iter_adjust > 0, run);
        if (!st) st = plan.launch_class(none, 0, 0, 0, run);
    }
    if (!st) st = cuda_status(cudaStreamBeginCapture(run, cudaStreamCaptureModeThreadLocal));
    if (!st) {
        const int est = plan.enqueue(iter_adjust, run);
        const int cst = cuda_status(cudaStreamEndCapture(run, &graph));
        st = est ? est : cst;
    }
    if (!st) st = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
    if (!st) st = cuda_status(cudaGraphLaunch(exec, run));
    std::vector<double> h(2 * (size_t)n_jobs * itmax);
    if (!st) st = cuda_status(cudaMemcpyAsync(h.data(), plan.d_sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, run));
    if (!st) st = cuda_status(cudaStreamSynchronize(run));
    if (!st && user) {
        st = cuda_status(cudaEventRecord(ev, run));
        if (!st) st = cuda_status(cudaStreamWaitEvent(user, ev, 0));
    }
    cleanup();
    if (st) return st;

    int worst = MCUBES_OK;
    for (int j = 0; j < n_jobs; ++j) {
        const Problem &p = plan.pb[j];
        const double *sj = h.data() + 2 * (size_t)itmax * j;
        combine_job(sj, itmax, (double)p.m, &out[j]);
        out[j].iters_done = itmax;
        out[j].samples_per_iter = p.m * p.p;
        if (out[j].status) worst = out[j].status;
        if (iter_out)
            for (int it = 0; it < itmax; ++it) {
                iter_out[(2 * (size_t)itmax) * j + 2 * it] = sj[2 * it] / (double)p.m;
                iter_out[(2 * (size_t)itmax) * j + 2 * it + 1] = sj[2 * it + 1] / ((double)p.m * (double)p.m);
            }
    }
    return worst;
}

extern "C" int mcubes_tune_batch(int n_jobs, const mcubes_job *jobs, int precision, mcubes_batch_tuning *out)
{
    int st = check_jobs(n_jobs, jobs);
    if (!out) st = MCUBES_ERR_INVALID_ARG;
    if (st) return st;
    std::memset(out, 0, sizeof(*out));
    Plan plan;
    if ((st = plan.init(n_jobs, jobs, 1, 1, precision))) return st;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)))) return st;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(s);
    };
    if (!st) st = cuda_status(cudaEventCreate(&e0));
    if (!st) st = cuda_status(cudaEventCreate(&e1));
    // uniform grids once
    if (!st) {
        batch_uniform_grids<<<n_jobs, 256, 0, s>>>(plan.d_gridptr[0], plan.d_dims, n_jobs);
        st = cuda_status(cudaGetLastError());
    }
    std::map<int, bool> dims;
    for (const auto &p : plan.pb) dims[p.d] = true;
    const int thr[2] = {128, 256};
    const int cpts[5] = {1, 2, 4, 8, 16};
    for (auto &kv : dims) {
        const int d = kv.first;
        float best = 1e30f;
        for (int ti = 0; ti < 2 && !st; ++ti)
            for (int ci = 0; ci < 5 && !st; ++ci)
                for (int hm = 0; hm < 2 && !st; ++hm) {
                    mcubes_batch_tuning cand;
                    std::memset(&cand, 0, sizeof(cand));
                    cand.block_threads[d] = thr[ti];
                    cand.cubes_per_thread[d] = cpts[ci];
                    cand.hist_mode[d] = hm;
                    if ((st = plan.tile(&cand))) break;
                    float total = 0.0f;
                    for (int rep = 0; rep < 2 && !st; ++rep) {   // rep 0 warms up
                        st = cuda_status(cudaMemsetAsync(plan.d_C, 0, sizeof(double) * plan.C_doubles, s));
                        if (!st) st = cuda_status(cudaEventRecord(e0, s));
                        for (const auto &c : plan.classes)
                            if (!st && c.d == d) st = plan.launch_class(c, 0, 0, 1, s);
                        if (!st) st = cuda_status(cudaEventRecord(e1, s));
                        if (!st) st = cuda_status(cudaEventSynchronize(e1));
                        float ms = 0.0f;
                        if (!st) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
                        if (rep == 1) total = ms;
                    }
                    if (!st && total < best) {
                        best = total;
                        out->block_threads[d] = thr[ti];
                        out->cubes_per_thread[d] = cpts[ci];
                        out->hist_mode[d] = hm;
                    }
                }
    }
    cleanup();
    return st;
}
