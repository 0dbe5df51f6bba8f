// Batched runs (od_create_batch ... od_destroy_batch): many independent runs of uneven
// ion count advanced by one persistent launch per step (k_batch_step, od_batch.cu).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "od_host.h"

using namespace od;
using namespace od::host;

struct od_batch {
    std::vector<od_handle*> runs;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    RunDesc* d_runs = nullptr;
    int2* d_tasks = nullptr;
    int2* d_tasks_f = nullptr;          // tuning: pair units, then kick tiles
    unsigned long long* d_done = nullptr;
    unsigned long long* d_done_f = nullptr;  // phase counters of the tuning launches
    BatchCtrl* d_bc = nullptr;
    BatchCtrl* d_bc_f = nullptr;
    long long T = 0, T_f = 0;
    int4 phase_end{0, 0, 0, 0}, phase_end_f{0, 0, 0, 0};
    int ipt = 2, jc = 4096, grid = 1, sms = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    long long host_step = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(od_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return code;
}

#define OD_BCK(b, call)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? OD_ENOMEM : OD_ECUDA,                  \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// apply the batch pair plan (ipt, jc) to every run and rebuild the task lists
int batch_build(od_batch* b)
{
    const int R = (int)b->runs.size();
    std::vector<RunDesc> desc(R);
    std::vector<int2> tA, tF, tK, tD;
    for (int r = 0; r < R; ++r) {
        od_handle* h = b->runs[r];
        h->F = batch_plan(h->P.N, b->ipt, b->jc);
        attach_sums(h, h->F);
        h->P.n_pad = h->F.n_pad;
        if (h->F.n_pad > h->npad_cap) return bfail(b, OD_EOVERFLOW, "padded ion count exceeds a run's buffer");
        int rc = ensure_part(h);
        if (rc) return bfail(b, rc, h->err);
        rc = launch_fpos(h->P, h->B, (int)(h->host_step & 1), b->stream);
        if (rc) return bfail(b, OD_ECUDA, "batch: position refresh failed");
        desc[r].P = h->P;
        desc[r].B = h->B;
        desc[r].F = h->F;
        desc[r].nA = (h->P.N + BATCH_TILE - 1) / BATCH_TILE;
        desc[r].nK = desc[r].nA;
        if (desc[r].nA > h->scan_tiles_cap || desc[r].nK > h->nb_cap)
            return bfail(b, OD_EINVAL, "batch: run " + std::to_string(r) + " has more scan or kick tiles than its buffers");
        for (int i = 0; i < desc[r].nA; ++i) tA.push_back(make_int2(r, i));
        for (long long u = 0; u < h->F.U; ++u) tF.push_back(make_int2(r, (int)u));
        for (int i = 0; i < desc[r].nK; ++i) tK.push_back(make_int2(r, i));
        tD.push_back(make_int2(r, 0));
    }
    std::vector<int2> all;
    all.insert(all.end(), tA.begin(), tA.end());
    all.insert(all.end(), tF.begin(), tF.end());
    all.insert(all.end(), tK.begin(), tK.end());
    all.insert(all.end(), tD.begin(), tD.end());
    b->phase_end = make_int4((int)tA.size(), (int)(tA.size() + tF.size()), (int)(tA.size() + tF.size() + tK.size()),
                             (int)all.size());
    b->T = (long long)all.size();
    std::vector<int2> fk(tF);
    fk.insert(fk.end(), tK.begin(), tK.end());
    b->phase_end_f = make_int4(0, (int)tF.size(), (int)fk.size(), (int)fk.size());
    b->T_f = (long long)fk.size();
    cudaFree(b->d_runs);
    cudaFree(b->d_tasks);
    cudaFree(b->d_tasks_f);
    b->d_runs = nullptr;
    b->d_tasks = b->d_tasks_f = nullptr;
    OD_BCK(b, cudaMalloc(&b->d_runs, sizeof(RunDesc) * R));
    OD_BCK(b, cudaMalloc(&b->d_tasks, sizeof(int2) * std::max<size_t>(all.size(), 1)));
    OD_BCK(b, cudaMalloc(&b->d_tasks_f, sizeof(int2) * std::max<size_t>(fk.size(), 1)));
    OD_BCK(b, cudaMemcpyAsync(b->d_runs, desc.data(), sizeof(RunDesc) * R, cudaMemcpyHostToDevice, b->stream));
    OD_BCK(b, cudaMemcpyAsync(b->d_tasks, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice, b->stream));
    if (!fk.empty())
        OD_BCK(b, cudaMemcpyAsync(b->d_tasks_f, fk.data(), sizeof(int2) * fk.size(), cudaMemcpyHostToDevice, b->stream));
    b->grid = (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms, b->T));
    OD_BCK(b, cudaStreamSynchronize(b->stream));
    b->graph_ok = false;
    return OD_OK;
}

void batch_free(od_batch* b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (od_handle* h : b->runs) {
        free_all(h);
        delete h;
    }
    cudaFree(b->d_runs);
    cudaFree(b->d_tasks);
    cudaFree(b->d_tasks_f);
    cudaFree(b->d_done);
    cudaFree(b->d_done_f);
    cudaFree(b->d_bc);
    cudaFree(b->d_bc_f);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int batch_check(od_batch* b)
{
    BatchCtrl bc;
    OD_BCK(b, cudaMemcpyAsync(&bc, b->d_bc, sizeof(bc), cudaMemcpyDeviceToHost, b->stream));
    OD_BCK(b, cudaStreamSynchronize(b->stream));
    if (bc.err & ERR_TIMEOUT) return bfail(b, OD_ETIMEOUT, "batch: a task's dependency wait hit its limit");
    for (size_t r = 0; r < b->runs.size(); ++r) {
        const int rc = read_error_word(b->runs[r]);
        if (rc) return bfail(b, rc, "run " + std::to_string(r) + ": " + b->runs[r]->err);
    }
    return OD_OK;
}

}  // namespace

extern "C" {

int od_create_batch(const od_params* ps, int32_t R, od_batch** out)
{
    if (!out || !ps || R < 1) return bfail(nullptr, OD_EINVAL, "bad batch arguments");
    *out = nullptr;
    for (int r = 0; r < R; ++r) {
        std::string msg;
        const int rc = validate(ps + r, msg);
        if (rc) return bfail(nullptr, rc, "run " + std::to_string(r) + ": " + msg);
        if (ps[r].flags & OD_F_FLUX_INJECT)
            return bfail(nullptr, OD_EINVAL, "run " + std::to_string(r) + ": batched runs keep a fixed ion count");
        if (ps[r].flags & OD_F_FP64_PAIRS)
            return bfail(nullptr, OD_EINVAL, "run " + std::to_string(r) + ": the FP64 study kernel runs alone");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bfail(nullptr, OD_ENODEV, "no CUDA device");
    od_batch* b = new od_batch();
    int rc = OD_OK;
    auto fail_out = [&](int code) {
        g_batch_error = b->err;
        batch_free(b);
        delete b;
        return code;
    };
    if (ps[0].cuda_stream) {
        b->stream = (cudaStream_t)ps[0].cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        b->err = "stream creation failed";
        return fail_out(OD_ECUDA);
    } else {
        b->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int r = 0; r < R; ++r) {
        od_params p = ps[r];
        p.cuda_stream = b->stream;
        od_handle* h = new od_handle();
        h->batch_member = true;
        rc = create_impl(&p, h);
        if (rc) {
            b->err = "run " + std::to_string(r) + ": " + h->err;
            free_all(h);
            delete h;
            return fail_out(rc);
        }
        h->batch_member = true;
        h->own_stream = false;
        b->runs.push_back(h);
    }
    if (cudaMalloc(&b->d_done, sizeof(unsigned long long) * 3 * R) != cudaSuccess ||
        cudaMalloc(&b->d_done_f, sizeof(unsigned long long) * 3 * R) != cudaSuccess ||
        cudaMalloc(&b->d_bc, sizeof(BatchCtrl)) != cudaSuccess || cudaMalloc(&b->d_bc_f, sizeof(BatchCtrl)) != cudaSuccess ||
        cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
        b->err = "batch allocation failed";
        return fail_out(OD_ENOMEM);
    }
    cudaMemsetAsync(b->d_done, 0, sizeof(unsigned long long) * 3 * R, b->stream);
    cudaMemsetAsync(b->d_bc, 0, sizeof(BatchCtrl), b->stream);
    rc = batch_build(b);
    if (rc) return fail_out(rc);
    *out = b;
    return OD_OK;
}

int od_batch_step(od_batch* b, int64_t n)
{
    if (!b || n < 0) return bfail(b, OD_EINVAL, "bad batch or step count");
    if (n == 0) return OD_OK;
    for (od_handle* h : b->runs) {
        const int rc = ensure_series(h, h->host_step + n);
        if (rc) return bfail(b, rc, h->err);
    }
    if (!b->graph_ok) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->gexec = nullptr;
        b->graph = nullptr;
        OD_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int lrc = launch_batch(b->ipt, b->grid, b->d_runs, b->d_tasks, b->phase_end, b->T, b->d_bc, b->d_done,
                                     (int)b->runs.size(), SPIN_LIMIT, 0, b->stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (lrc) return bfail(b, OD_ECUDA, std::string("batch launch: ") + cudaGetErrorString((cudaError_t)lrc));
        if (e != cudaSuccess) return bfail(b, OD_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
        b->graph = g;
        OD_BCK(b, cudaGraphInstantiate(&b->gexec, g, 0));
        b->graph_ok = true;
    }
    for (int64_t s = 0; s < n; ++s) OD_BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    for (od_handle* h : b->runs) h->host_step += n;
    b->host_step += n;
    return batch_check(b);
}

od_handle* od_batch_run(od_batch* b, int32_t r)
{
    if (!b || r < 0 || r >= (int)b->runs.size()) return nullptr;
    return b->runs[r];
}

int od_batch_size(const od_batch* b) { return b ? (int)b->runs.size() : 0; }

// one tuning launch of the current plan: every run's pair units, then its kick tiles in
// forces-only mode (fresh counters per configuration)
static int batch_tune_launch(od_batch* b, int grid)
{
    const int lrc = launch_batch(b->ipt, grid, b->d_runs, b->d_tasks_f, b->phase_end_f, b->T_f, b->d_bc_f,
                                 b->d_done_f, (int)b->runs.size(), SPIN_LIMIT, 1, b->stream);
    return lrc ? bfail(b, OD_ECUDA, "batch tune launch failed") : OD_OK;
}

int od_batch_tune(od_batch* b, int reps, double* ms, int* best_ipt, int* best_jc)
{
    if (!b || reps < 1) return bfail(b, OD_EINVAL, "bad batch or repetition count");
    static const int ipts[3] = {2, 4, 8};
    static const int jcs[4] = {2048, 4096, 8192, 0};  // 0: symmetric tile pairs
    double best = 1e300;
    int bi = b->ipt, bj = b->jc;
    const int R = (int)b->runs.size();
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 4; ++c) {
            b->ipt = ipts[a];
            b->jc = jcs[c];
            int rc = batch_build(b);
            if (rc) return rc;
            OD_BCK(b, cudaMemsetAsync(b->d_bc_f, 0, sizeof(BatchCtrl), b->stream));
            OD_BCK(b, cudaMemsetAsync(b->d_done_f, 0, sizeof(unsigned long long) * 3 * R, b->stream));
            const int grid = (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms, b->T_f));
            if ((rc = batch_tune_launch(b, grid))) return rc;
            OD_BCK(b, cudaEventRecord(b->e0, b->stream));
            for (int i = 0; i < reps; ++i)
                if ((rc = batch_tune_launch(b, grid))) return rc;
            OD_BCK(b, cudaEventRecord(b->e1, b->stream));
            OD_BCK(b, cudaEventSynchronize(b->e1));
            float t = 0.f;
            OD_BCK(b, cudaEventElapsedTime(&t, b->e0, b->e1));
            if (ms) ms[a * 4 + c] = t / reps;
            if (t / reps < best) {
                best = t / reps;
                bi = ipts[a];
                bj = jcs[c];
            }
        }
    b->ipt = bi;
    b->jc = bj;
    int rc = batch_build(b);
    if (rc) return rc;
    // the accelerations left by the timing belong to other plans: evaluate them again
    // with the chosen one
    OD_BCK(b, cudaMemsetAsync(b->d_bc_f, 0, sizeof(BatchCtrl), b->stream));
    OD_BCK(b, cudaMemsetAsync(b->d_done_f, 0, sizeof(unsigned long long) * 3 * R, b->stream));
    if ((rc = batch_tune_launch(b, (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms,
                                                                            b->T_f)))))
        return rc;
    if ((rc = batch_check(b))) return rc;
    if (best_ipt) *best_ipt = bi;
    if (best_jc) *best_jc = bj;
    return OD_OK;
}

int od_batch_set_config(od_batch* b, int ipt, int jc)
{
    if (!b || (ipt != 2 && ipt != 4 && ipt != 8) || (jc != 0 && jc < 256))
        return bfail(b, OD_EINVAL, "bad batch configuration");
    b->ipt = ipt;
    b->jc = jc;
    return batch_build(b);
}

void od_destroy_batch(od_batch* b)
{
    if (!b) return;
    batch_free(b);
    delete b;
}

const char* od_batch_last_error(const od_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"

