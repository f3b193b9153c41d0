// Host side of libbs: contexts, device buffers under a memory budget, the
// integer planner (canonicalisation of a permanent / minors problem), launch
// sequencing on the context stream, the Clifford & Clifford driver loop, and
// the C ABI declared in include/bs.h.
//
// Canonicalisation (Sec. 2.2, Eq. bbfgrepeated):
//   * rows / columns with multiplicity 0 are dropped; sum(M) = sum(N) = n is
//     checked (minors: sum(M) = sum(N) - 1);
//   * permanents are evaluated in the orientation (A or A^T, perm(A) =
//     perm(A^T)) whose row multiplicities give fewer addends;
//   * the pinned row (delta = +1, "always treated with a multiplicity of 1")
//     is a row of smallest multiplicity; if that multiplicity is M_p > 1 its
//     other M_p - 1 copies become a digit of radix M_p (the paper suggests
//     moving a non-repeated row to the top; any choice gives the same sum);
//   * digits: multiplicity-1 rows first (binary, fastest), then repeated rows
//     by increasing multiplicity;
//   * repeated columns are expanded, so every product column has
//     multiplicity 1 and the product length is n (minors: n + 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bs.h"
#include "bs_job.h"
#include "gray.h"
#include "kernels.h"
#include "plan.h"
#include "sample.h"

namespace {

using bs::fail;

#define BS_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(BS_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                        \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

// control block layout (unsigned long long slots)
constexpr int kMaxGroups = 64;
constexpr int kCtlStatus = kMaxGroups;                          // int status word (in a 64-bit slot)
constexpr int kCtlTotal = kMaxGroups + 1;                       // sampler task totals, one per precision
constexpr int kCtlCounter = kCtlTotal + BS_NPREC;                // sampler work counters, one per precision
constexpr int kCtlStats = kCtlCounter + BS_NPREC;                // [addends, flops] per precision
constexpr int kCtlListLen = kCtlStats + 2 * BS_NPREC;            // ints: sampler list lengths
constexpr int kCtlSlots = kCtlListLen + 8;

struct Timed {
    cudaEvent_t e0, e1;
    int prec;  // BS_PREC_* of the timed walk
};

}  // namespace

struct bs_ctx {
    int device = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    DevBuf src, jobs, meta, data64, data32, partials, out, out_lo, ctl;
    DevBuf cc_inputs, cc_cols, cc_rows, cc_jobs, cc_meta, cc_data, cc_partials, cc_minors, cc_out, cc_U, cc_lists,
        cc_args;
    // captured sampler step loop (one batch), replayed while its key matches
    bool use_graphs = true;
    cudaGraphExec_t cc_exec = nullptr;
    std::vector<uint64_t> cc_key;
    uint64_t cc_graph_kernels = 0;
    // walk timing events captured into the sampler graph (profiling): owned
    // by the graph, re-recorded at every replay and read before the next one
    std::vector<Timed> cc_graph_timed;
    bool cc_timing_pending = false;
    // captured device sequence of the last device-pointer batch, replayed
    // while the batch's shapes, multiplicities, offsets, mode, chunk caps and
    // deadline, its device pointers and the context buffers are unchanged
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<int64_t> batch_key;
    const void* batch_src = nullptr;
    void* batch_out = nullptr;
    void* batch_out_lo = nullptr;
    std::vector<int64_t> single_last_key;  // key of the last single call (capture on a repeat)
    uint64_t batch_gen = 0;
    uint64_t batch_walks = 0, batch_kernels = 0, batch_adds[BS_NPREC] = {}, batch_flops[BS_NPREC] = {};
    // bumped whenever the job/metadata buffers are rewritten or any buffer
    // is reallocated (a captured graph refers to them)
    uint64_t buf_gen = 1;
    // two pinned staging buffers, used in turn: a buffer is reused only after
    // the copy out of it (stage_ev) has finished, so staging one upload never
    // waits for the copy just enqueued from the other
    void* h_stage[2] = {nullptr, nullptr};
    size_t h_stage_n[2] = {0, 0};
    int stage_cur = 0;
    void* h_back = nullptr;  // pinned read-back buffer of single calls
    size_t h_back_n = 0;
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    double deadline_s = 0.0;
    int log2max[BS_NPREC] = {bs_default_log2max(BS_PREC_FP64), bs_default_log2max(BS_PREC_FP32),
                             bs_default_log2max(BS_PREC_DF)};  // chunk-length caps, indexed by precision (= bs_mode)
    float mixed_log2_tol = BS_MIXED_LOG2_TOL_DEFAULT;  // MIXED precision rule threshold
    bool profiling = false;
    std::vector<Timed> timed;
    std::vector<double> walk_log;  // per-launch walk durations not yet read
    bs_stats stats{};
    std::mutex mu;
};

namespace {

int ensure(bs_ctx* c, DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return BS_OK;
    size_t want = std::max(bytes, b.n + b.n / 4);
    if (c->budget && c->used - b.n + want > c->budget) {
        want = bytes;
        if (c->used - b.n + want > c->budget)
            return fail(BS_ENOMEM, "device memory budget exceeded: need %zu more bytes (budget %zu, in use %zu)",
                        want - b.n, c->budget, c->used);
    }
    c->buf_gen++;
    if (b.p) {
        cudaFree(b.p);
        c->used -= b.n;
        b.p = nullptr;
        b.n = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BS_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.n = want;
    c->used += want;
    return BS_OK;
}

void release(bs_ctx* c, DevBuf& b) {
    if (b.p) cudaFree(b.p);
    c->used -= b.n;
    b.p = nullptr;
    b.n = 0;
}

// The next of the two pinned staging buffers, at least `bytes` long; waits
// first for the last copy recorded out of it (stage_ev of that buffer).
// Callers record c->stage_ev[c->stage_cur] after enqueueing their copy.
void* stage(bs_ctx* c, size_t bytes) {
    const int b = c->stage_cur ^ 1;
    if (c->stage_ev[b]) cudaEventSynchronize(c->stage_ev[b]);
    c->stage_cur = b;
    if (c->h_stage_n[b] < bytes) {
        if (c->h_stage[b]) cudaFreeHost(c->h_stage[b]);
        size_t want = std::max(bytes, c->h_stage_n[b] * 2);
        if (cudaHostAlloc(&c->h_stage[b], want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            c->h_stage[b] = nullptr;
            c->h_stage_n[b] = 0;
            return nullptr;
        }
        c->h_stage_n[b] = want;
    }
    return c->h_stage[b];
}

using bs::IntPlan;
using bs::plan_job;
using bs::first_product_col;

// ------------------------------------------------------------------ launcher
struct JobIn {
    const IntPlan* p;
    int64_t src_off;
    int src_ld;
    int out_index;
};

// Reads the walk durations of the last profiled sampler-graph replay into the
// statistics (waits for that replay to finish).
void harvest_graph_timing(bs_ctx* c) {
    if (!c->cc_timing_pending || c->cc_graph_timed.empty()) return;
    cudaEventSynchronize(c->cc_graph_timed.back().e1);
    for (auto& t : c->cc_graph_timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
            c->stats.walk_ms[t.prec] += ms;
            c->stats.timed_launches[t.prec]++;
            c->walk_log.push_back(ms);
        } else {
            cudaGetLastError();  // leave no stale error for the next launch check
        }
    }
    c->cc_timing_pending = false;
}

void drop_graph_timing(bs_ctx* c) {
    for (auto& t : c->cc_graph_timed) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    c->cc_graph_timed.clear();
    c->cc_timing_pending = false;
}

// Records a timing event on the context stream; while the stream is being
// captured the record becomes an event-record node of the graph (a plain
// record there would only order work inside the graph).
cudaError_t record_timing_event(bs_ctx* c, cudaEvent_t e) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (c->stream != nullptr) {
        cudaError_t err = cudaStreamIsCapturing(c->stream, &cap);
        if (err != cudaSuccess) return err;
    }
    return cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal)
                                                : cudaEventRecord(e, c->stream);
}

int record_walk_start(bs_ctx* c, cudaEvent_t* e0) {
    *e0 = nullptr;
    if (!c->profiling) return BS_OK;
    BS_CUDA(cudaEventCreate(e0));
    const cudaError_t e = record_timing_event(c, *e0);
    if (e != cudaSuccess) {
        cudaEventDestroy(*e0);
        *e0 = nullptr;
        BS_CUDA(e);
    }
    return BS_OK;
}

// Takes ownership of e0 (recorded by record_walk_start).
int record_walk_end(bs_ctx* c, cudaEvent_t e0, int prec) {
    if (!c->profiling || !e0) return BS_OK;
    cudaEvent_t e1;
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        e = record_timing_event(c, e1);
        if (e != cudaSuccess) cudaEventDestroy(e1);
    }
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        BS_CUDA(e);
    }
    c->timed.push_back({e0, e1, prec});
    return BS_OK;
}

int launch_walk(bs_ctx* c, const bs::WalkArgs& a, int prec, int kind) {
    cudaEvent_t e0;
    int rc = record_walk_start(c, &e0);
    if (rc) return rc;
    cudaError_t e;
    if (prec == BS_PREC_DF)
        e = kind == BS_KIND_PERM ? bs::launch_walk_df_perm(a, c->stream) : bs::launch_walk_df_minors(a, c->stream);
    else if (prec == BS_PREC_FP32)
        e = kind == BS_KIND_PERM ? bs::launch_walk_fp32_perm(a, c->stream) : bs::launch_walk_fp32_minors(a, c->stream);
    else
        e = kind == BS_KIND_PERM ? bs::launch_walk_fp64_perm(a, c->stream) : bs::launch_walk_fp64_minors(a, c->stream);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(BS_ECUDA, "walk launch failed: %s", cudaGetErrorString(e));
    }
    c->stats.walk_launches++;
    c->stats.kernel_launches++;
    return record_walk_end(c, e0, prec);
}

// The MIXED mode's kernels for jobs that fail the FP32 rule.
constexpr int kMixedFallback = BS_MIXED_FALLBACK_PREC;

// Precision of a job planned under `mode` (rule_fp32: whether the MIXED
// rule admits FP32).
int job_prec(bs_mode mode, int rule_fp32) {
    if (mode == BS_DF64) return BS_PREC_DF;
    if (mode == BS_MIXED) return rule_fp32 ? BS_PREC_FP32 : kMixedFallback;
    return BS_PREC_FP64;
}

// Data arena of a precision: FP32 jobs in complex floats (data32), FP64 and
// DF jobs in 16-byte units (data64).
inline int arena_of(int prec) { return prec == BS_PREC_FP32 ? 1 : 0; }

bool valid_mode(bs_mode mode) { return mode == BS_FP64 || mode == BS_MIXED || mode == BS_DF64; }

// A planned and uploaded set of jobs: what the device sequence needs.
struct Prepared {
    struct Group {
        size_t first, last;
        int prec, kind, kmax;
        unsigned long long tasks;
    };
    std::vector<Group> groups;
    size_t njobs = 0;
    size_t pbeg[BS_NPREC + 1] = {};  // jobs [pbeg[p], pbeg[p + 1]) have precision p
    int max_cols = 1;
    uint64_t adds[BS_NPREC] = {}, flops[BS_NPREC] = {};
};

// Host half of a walk: plan every job (precision, chunking, groups of equal
// precision, kind and bucket, largest jobs first), size the device buffers
// and upload the job descriptors and metadata.
int plan_upload(bs_ctx* c, std::vector<JobIn>& ins, bs_mode mode, Prepared& P) {
    struct Row {
        JobIn in;
        int prec, kind, bucket, log2L, cpt, ncols, reseed;
        uint32_t ntasks;
    };
    std::vector<Row> rows;
    std::vector<double> q_work(BS_MIXED_QMAX + 1);
    for (auto& in : ins) {
        if (in.p->trivial) continue;
        Row r;
        r.in = in;
        int rule = 0;
        if (mode == BS_MIXED) {
            // the rule needs the chunk length the FP32 kernel would use
            const int cpt32 = bs_chunks_per_task(in.p->kind, BS_PREC_FP32, in.p->K);
            const int l32 = bs_choose_log2L_single(in.p->C, cpt32, c->log2max[BS_PREC_FP32], BS_TARGET_TASKS_SINGLE_FP32);
            rule = bs_mixed_fp32_plan(in.p->radix, in.p->nrows, in.p->pinned_m, in.p->K, in.p->n, l32,
                                      c->mixed_log2_tol, q_work.data());
        }
        r.prec = job_prec(mode, rule != 0);
        r.reseed = r.prec == BS_PREC_FP32 && rule == 2 ? BS_FP32_RESEED_LOG2 : 0;
        r.kind = in.p->kind;
        r.bucket = r.prec == BS_PREC_DF ? (in.p->K + 7) >> 3 : (in.p->K + 3) >> 2;
        r.cpt = bs_chunks_per_task(r.kind, r.prec, in.p->K);
        r.log2L = bs_choose_log2L_single(in.p->C, r.cpt, c->log2max[r.prec],
                                         r.prec == BS_PREC_FP32 ? BS_TARGET_TASKS_SINGLE_FP32 : BS_TARGET_TASKS_SINGLE);
        uint64_t per = (uint64_t)r.cpt << r.log2L;
        r.ntasks = (uint32_t)((in.p->C + per - 1) / per);
        r.ncols = r.kind == BS_KIND_PERM ? 1 : in.p->K;
        rows.push_back(r);
    }
    P = Prepared();
    if (rows.empty()) return BS_OK;
    // groups of equal (precision, kind, bucket); largest jobs first inside
    std::stable_sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
        if (a.prec != b.prec) return a.prec < b.prec;
        if (a.kind != b.kind) return a.kind < b.kind;
        if (a.bucket != b.bucket) return a.bucket < b.bucket;
        return a.in.p->C > b.in.p->C;
    });
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < rows.size();) {
        size_t j = i;
        while (j < rows.size() && rows[j].prec == rows[i].prec && rows[j].kind == rows[i].kind &&
               rows[j].bucket == rows[i].bucket)
            ++j;
        groups.push_back({i, j});
        i = j;
    }
    if ((int)groups.size() > kMaxGroups) return fail(BS_EINVAL, "too many kernel groups");
    std::vector<bs_job> jobs(rows.size());
    std::vector<int> meta;
    int64_t data_off[2] = {0, 0}, part_off = 0;
    int& max_cols = P.max_cols;
    uint64_t* adds = P.adds;
    uint64_t* flops = P.flops;
    for (auto& g : groups) {
        uint64_t tb = 0;
        for (size_t i = g.first; i < g.second; ++i) {
            const Row& r = rows[i];
            const IntPlan& p = *r.in.p;
            bs_job& jb = jobs[i];
            std::memset(&jb, 0, sizeof(jb));
            jb.C = p.C;
            jb.task_begin = tb;
            jb.ntasks = r.ntasks;
            jb.K = p.K;
            jb.nrows = p.nrows;
            jb.nbin = p.nbin;
            jb.kind = r.kind;
            jb.log2L = r.log2L;
            jb.out_index = r.in.out_index;
            jb.n = p.n;
            jb.normalize = r.prec != BS_PREC_FP64 ? 1 : 0;
            jb.prec = r.prec;
            jb.data_off = data_off[arena_of(r.prec)];
            jb.meta_off = (int64_t)meta.size();
            jb.partial_off = part_off;
            jb.src_off = r.in.src_off;
            jb.src_ld = r.in.src_ld;
            jb.src_trans = p.trans ? 1 : 0;
            jb.formula = p.formula;
            jb.reseed_log2 = r.reseed;
            meta.insert(meta.end(), p.radix, p.radix + p.nrows);
            meta.insert(meta.end(), p.digit_src, p.digit_src + p.nrows);
            meta.insert(meta.end(), p.col_src, p.col_src + p.K);
            meta.insert(meta.end(), (size_t)p.K, 0);
            meta.push_back(p.pinned_src);
            meta.push_back(0);                                           // pad to 8 bytes
            meta.insert(meta.end(), (size_t)2 * (p.nrows + p.n), 0);     // binomial table (pack kernel)
            data_off[arena_of(r.prec)] += (int64_t)(1 + p.nrows) * BS_ROW_STRIDE_P(p.K, r.prec);
            part_off += (int64_t)r.ntasks * r.ncols;
            tb += r.ntasks;
            max_cols = std::max(max_cols, r.ncols);
            adds[r.prec] += p.C;
            flops[r.prec] += p.C * (uint64_t)bs_flops_per_addend(p.K, r.kind);
        }
    }
    const size_t jobs_b = jobs.size() * sizeof(bs_job), meta_b = meta.size() * sizeof(int);
    int rc;
    if ((rc = ensure(c, c->jobs, jobs_b))) return rc;
    if ((rc = ensure(c, c->meta, meta_b))) return rc;
    if ((rc = ensure(c, c->data64, (size_t)data_off[0] * 16))) return rc;
    if ((rc = ensure(c, c->data32, (size_t)data_off[1] * 8))) return rc;
    if ((rc = ensure(c, c->partials, (size_t)part_off * sizeof(bs_zdd)))) return rc;
    if ((rc = ensure(c, c->ctl, kCtlSlots * 8))) return rc;
    char* h = static_cast<char*>(stage(c, jobs_b + meta_b));
    if (!h) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    std::memcpy(h, jobs.data(), jobs_b);
    std::memcpy(h + jobs_b, meta.data(), meta_b);
    BS_CUDA(cudaMemcpyAsync(c->jobs.p, h, jobs_b, cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaMemcpyAsync(c->meta.p, h + jobs_b, meta_b, cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaEventRecord(c->stage_ev[c->stage_cur], c->stream));
    c->buf_gen++;
    P.njobs = rows.size();
    // jobs are sorted by precision: FP64, then FP32, then DF
    for (int q = 0; q <= BS_NPREC; ++q) {
        size_t at = 0;
        while (at < rows.size() && rows[at].prec < q) ++at;
        P.pbeg[q] = at;
    }
    for (auto& g : groups) {
        Prepared::Group G;
        G.first = g.first;
        G.last = g.second;
        G.prec = rows[g.first].prec;
        G.kind = rows[g.first].kind;
        G.kmax = 0;
        G.tasks = 0;
        for (size_t i = g.first; i < g.second; ++i) {
            G.tasks += rows[i].ntasks;
            G.kmax = std::max(G.kmax, rows[i].in.p->K);
        }
        P.groups.push_back(G);
    }
    return BS_OK;
}

// Device half: counters, pack, one walk launch per group, reduce; nothing
// that synchronises, so it can be captured into a graph.
int enqueue_device(bs_ctx* c, const Prepared& P, const double2* d_src, double2* d_out, double2* d_out_lo) {
    int rc;
    // counters, totals and status; the statistics slots are cleared only by
    // bs_ctx_reset_stats
    BS_CUDA(cudaMemsetAsync(c->ctl.p, 0, kCtlStats * 8, c->stream));
    BS_CUDA(cudaMemsetAsync(static_cast<unsigned long long*>(c->ctl.p) + kCtlListLen, 0, (kCtlSlots - kCtlListLen) * 8, c->stream));
    const bs_job* djobs = static_cast<const bs_job*>(c->jobs.p);
    for (int prec = 0; prec < BS_NPREC; ++prec) {
        const size_t lo = P.pbeg[prec], hi = P.pbeg[prec + 1];
        if (hi == lo) continue;
        cudaError_t e = bs::launch_pack(djobs + lo, (int)(hi - lo), d_src, static_cast<int*>(c->meta.p),
                                        arena_of(prec) ? c->data32.p : c->data64.p, prec, c->stream);
        if (e != cudaSuccess) return fail(BS_ECUDA, "pack launch failed: %s", cudaGetErrorString(e));
        c->stats.kernel_launches++;
    }
    unsigned long long* ctl = static_cast<unsigned long long*>(c->ctl.p);
    for (size_t gi = 0; gi < P.groups.size(); ++gi) {
        const Prepared::Group& g = P.groups[gi];
        bs::WalkArgs w;
        std::memset(&w, 0, sizeof(w));
        w.jobs = djobs + g.first;
        w.njobs = (int)(g.last - g.first);
        w.data = arena_of(g.prec) ? c->data32.p : c->data64.p;
        w.meta = static_cast<const int*>(c->meta.p);
        w.partials = static_cast<bs_zdd*>(c->partials.p);
        w.total_tasks = g.tasks;
        w.counter = ctl + gi;
        w.status = reinterpret_cast<int*>(ctl + kCtlStatus);
        w.deadline_rel_ns = c->deadline_s > 0 ? (unsigned long long)(c->deadline_s * 1e9) : 0ull;
        w.max_K = g.kmax;
        if ((rc = launch_walk(c, w, g.prec, g.kind))) return rc;
    }
    {
        cudaError_t e = bs::launch_reduce(djobs, (int)P.njobs, static_cast<const bs_zdd*>(c->partials.p),
                                          static_cast<const int*>(c->meta.p), d_out, d_out_lo, P.max_cols, c->stream);
        if (e != cudaSuccess) return fail(BS_ECUDA, "reduce launch failed: %s", cudaGetErrorString(e));
        c->stats.kernel_launches++;
    }
    return BS_OK;
}

int run_jobs(bs_ctx* c, std::vector<JobIn>& ins, const double2* d_src, bs_mode mode, double2* d_out,
             double2* d_out_lo) {
    Prepared P;
    int rc = plan_upload(c, ins, mode, P);
    if (rc || P.njobs == 0) return rc;
    if ((rc = enqueue_device(c, P, d_src, d_out, d_out_lo))) return rc;
    for (int p = 0; p < BS_NPREC; ++p) {
        c->stats.addends[p] += P.adds[p];
        c->stats.addend_flops[p] += P.flops[p];
    }
    return BS_OK;
}

int check_status(bs_ctx* c) {
    if (!c->ctl.p) return BS_OK;
    int st = 0;
    BS_CUDA(cudaMemcpy(&st, static_cast<unsigned long long*>(c->ctl.p) + kCtlStatus, sizeof(int),
                       cudaMemcpyDeviceToHost));
    if (st == BS_STATUS_TIMEOUT) return fail(BS_ETIMEOUT, "a walk kernel passed its deadline");
    if (st == BS_STATUS_BADJOB) return fail(BS_ECUDA, "a walk kernel received a job of the wrong bucket");
    return BS_OK;
}

// Reads nout results (hi, lo) and the walk status word back through one
// pinned buffer and one stream synchronisation.
int read_back_and_check(bs_ctx* c, double2* hi, double2* lo, int nout) {
    const size_t out_b = (size_t)nout * sizeof(double2);
    const size_t need = 2 * out_b + sizeof(unsigned long long);
    if (c->h_back_n < need) {
        if (c->h_back) cudaFreeHost(c->h_back);
        c->h_back = nullptr;
        c->h_back_n = 0;
        const size_t want = std::max(need, (size_t)4096);
        BS_CUDA(cudaHostAlloc(&c->h_back, want, cudaHostAllocDefault));
        c->h_back_n = want;
    }
    char* h = static_cast<char*>(c->h_back);
    BS_CUDA(cudaMemcpyAsync(h, c->out.p, out_b, cudaMemcpyDeviceToHost, c->stream));
    BS_CUDA(cudaMemcpyAsync(h + out_b, c->out_lo.p, out_b, cudaMemcpyDeviceToHost, c->stream));
    BS_CUDA(cudaMemcpyAsync(h + 2 * out_b, static_cast<unsigned long long*>(c->ctl.p) + kCtlStatus,
                            sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(BS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    std::memcpy(hi, h, out_b);
    std::memcpy(lo, h + out_b, out_b);
    int st = 0;
    std::memcpy(&st, h + 2 * out_b, sizeof(int));
    if (st == BS_STATUS_TIMEOUT) return fail(BS_ETIMEOUT, "a walk kernel passed its deadline");
    if (st == BS_STATUS_BADJOB) return fail(BS_ECUDA, "a walk kernel received a job of the wrong bucket");
    return BS_OK;
}

int sync_and_check(bs_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(BS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return check_status(c);
}

bool ok_ctx(bs_ctx* c) {
    if (!c) {
        fail(BS_EINVAL, "context is NULL");
        return false;
    }
    return true;
}

// Copies rows x cols of A (leading dimension ld) to the staging buffer at
// offset `at` (in complex elements), contiguous.
void copy_matrix(bs_c128* dst, const bs_c128* A, int rows, int cols, int ld) {
    for (int r = 0; r < rows; ++r) std::memcpy(dst + (size_t)r * cols, A + (size_t)r * ld, sizeof(bs_c128) * cols);
}

// Walks a validated batch whose sources sit at d_src (+ each item's offset)
// and writes item b to d_out[b].  The device sequence of the last batch is
// kept as a captured CUDA graph: a batch with the same key, the same device
// pointers and untouched context buffers replays it without planning,
// uploading or launching anew.  Eager when graphs are off, when profiling, on
// the legacy default stream and while the caller captures the stream.
int batch_walk(bs_ctx* c, std::vector<IntPlan>& plans, const std::vector<int64_t>& key,
                      const int64_t* a_offset, const int* cols, const double2* d_src, double2* d_out, bs_mode mode,
                      double2* d_out_lo, bool capture_on_repeat = false) {
    int rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (c->stream != nullptr) BS_CUDA(cudaStreamIsCapturing(c->stream, &cap));
    bool graphs = c->use_graphs && !c->profiling && c->stream != nullptr && c->stream != cudaStreamPerThread &&
                  cap == cudaStreamCaptureStatusNone;
    if (capture_on_repeat) {
        // single calls: a capture costs more than one eager run, so a key is
        // captured only when it repeats the previous single call's
        const bool repeat = c->single_last_key == key;
        if (!repeat) c->single_last_key = key;
        if (!repeat && !(c->batch_exec && c->batch_key == key)) graphs = false;
    }
    if (graphs && c->batch_exec && c->batch_gen == c->buf_gen && c->batch_src == d_src && c->batch_out == d_out &&
        c->batch_out_lo == d_out_lo && c->batch_key == key) {
        BS_CUDA(cudaGraphLaunch(c->batch_exec, c->stream));
        c->stats.walk_launches += c->batch_walks;
        c->stats.kernel_launches += c->batch_kernels;
        for (int p = 0; p < BS_NPREC; ++p) {
            c->stats.addends[p] += c->batch_adds[p];
            c->stats.addend_flops[p] += c->batch_flops[p];
        }
        return BS_OK;
    }
    std::vector<JobIn> ins;
    for (size_t b = 0; b < plans.size(); ++b)
        if (!plans[b].trivial) ins.push_back({&plans[b], a_offset[b], cols[b], (int)b});
    Prepared P;
    if ((rc = plan_upload(c, ins, mode, P))) return rc;
    if (P.njobs == 0) return BS_OK;
    if (!graphs) {
        if ((rc = enqueue_device(c, P, d_src, d_out, d_out_lo))) return rc;
    } else {
        const uint64_t w0 = c->stats.walk_launches, k0 = c->stats.kernel_launches;
        BS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_device(c, P, d_src, d_out, d_out_lo);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc ? rc : fail(BS_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(BS_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
        if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
        c->batch_exec = exec;
        c->batch_key = key;
        c->batch_gen = c->buf_gen;
        c->batch_src = d_src;
        c->batch_out = d_out;
        c->batch_out_lo = d_out_lo;
        c->batch_walks = c->stats.walk_launches - w0;
        c->batch_kernels = c->stats.kernel_launches - k0;
        for (int p = 0; p < BS_NPREC; ++p) {
            c->batch_adds[p] = P.adds[p];
            c->batch_flops[p] = P.flops[p];
        }
        BS_CUDA(cudaGraphLaunch(c->batch_exec, c->stream));
    }
    for (int p = 0; p < BS_NPREC; ++p) {
        c->stats.addends[p] += P.adds[p];
        c->stats.addend_flops[p] += P.flops[p];
    }
    return BS_OK;
}

// The MIXED threshold as a key entry (its bits).
static int64_t tol_key(const bs_ctx* c) {
    int32_t b = 0;
    std::memcpy(&b, &c->mixed_log2_tol, sizeof(b));
    return b;
}

// Graph-cache key of one job planned alone: everything the device sequence
// depends on besides the buffers (the plan's digits, sources and product
// columns, the source shape, mode, chunk caps and deadline).  The leading -1
// keeps it apart from every batch key (which starts with the item count).
static std::vector<int64_t> plan_key(const bs_ctx* c, const IntPlan& p, int rows, int cols, bs_mode mode) {
    int64_t dl = 0;
    std::memcpy(&dl, &c->deadline_s, sizeof(dl));
    std::vector<int64_t> k = {-1, (int64_t)p.kind, (int64_t)p.formula, (int64_t)p.n, (int64_t)p.K,
                              (int64_t)p.nrows, (int64_t)p.nbin, (int64_t)p.C, (int64_t)p.trans,
                              (int64_t)p.pinned_src, (int64_t)rows, (int64_t)cols, (int64_t)mode,
                              (int64_t)c->log2max[0], (int64_t)c->log2max[1], (int64_t)c->log2max[2], dl,
                              tol_key(c)};
    for (int j = 0; j < p.nrows; ++j) k.insert(k.end(), {(int64_t)p.radix[j], (int64_t)p.digit_src[j]});
    for (int j = 0; j < p.K; ++j) k.push_back(p.col_src[j]);
    return k;
}

// One planned job on a rows x cols host matrix: upload, walk, reduce, read
// back (hi, lo: one value per output column).  When the plan repeats the
// previous single call's, the device sequence is captured as a graph and
// replayed while it keeps repeating (only the matrix upload and the read-back
// run outside it).
int run_single(bs_ctx* c, const bs_c128* A, int rows, int cols, int ld, int kind, bs_mode mode, const IntPlan& p,
               std::vector<double2>& hi, std::vector<double2>& lo) {
    int rc;
    const int nout = kind == BS_KIND_PERM ? 1 : std::max(p.K, 1);
    hi.assign(nout, make_double2(0, 0));
    lo.assign(nout, make_double2(0, 0));
    if (p.trivial) {
        hi[0] = make_double2(1.0, 0.0);
        return BS_OK;
    }
    if (!A) return fail(BS_EINVAL, "matrix pointer is NULL");
    if (ld < cols) return fail(BS_EINVAL, "leading dimension %d < columns %d", ld, cols);
    std::lock_guard<std::mutex> lk(c->mu);
    BS_CUDA(cudaSetDevice(c->device));
    const size_t mat_b = (size_t)rows * cols * sizeof(bs_c128);
    if ((rc = ensure(c, c->src, mat_b))) return rc;
    if ((rc = ensure(c, c->out, nout * sizeof(double2)))) return rc;
    if ((rc = ensure(c, c->out_lo, nout * sizeof(double2)))) return rc;
    bs_c128* h = static_cast<bs_c128*>(stage(c, mat_b));
    if (!h) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    copy_matrix(h, A, rows, cols, ld);
    BS_CUDA(cudaMemcpyAsync(c->src.p, h, mat_b, cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaEventRecord(c->stage_ev[c->stage_cur], c->stream));
    std::vector<IntPlan> plans = {p};
    const int64_t off0 = 0;
    rc = batch_walk(c, plans, plan_key(c, p, rows, cols, mode), &off0, &cols, static_cast<const double2*>(c->src.p),
                    static_cast<double2*>(c->out.p), mode, static_cast<double2*>(c->out_lo.p), true);
    if (rc) return rc;
    return read_back_and_check(c, hi.data(), lo.data(), nout);
}

int single_job(bs_ctx* c, const bs_c128* A, int rows, int cols, int ld, const int* M, const int* N, int kind,
               bs_mode mode, IntPlan& p, std::vector<double2>& hi, std::vector<double2>& lo) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode %d", (int)mode);
    int rc = plan_job(rows, cols, M, N, kind, p);
    if (rc) return rc;
    return run_single(c, A, rows, cols, ld, kind, mode, p, hi, lo);
}

// ------------------------------------------------------------------ sampler
// The walk kernels a sampler step launches under `mode`, in launch order:
// MIXED runs the FP32 kernel and the fallback kernel, the others one each.
int sampler_precs(bs_mode mode, int* precs) {
    if (mode == BS_MIXED) {
        precs[0] = BS_PREC_FP32;
        precs[1] = kMixedFallback;
        return 2;
    }
    precs[0] = mode == BS_DF64 ? BS_PREC_DF : BS_PREC_FP64;
    return 1;
}

// Walk launches per sampler batch (steps 2..n).
uint64_t kernels_walks(int n, bs_mode mode) {
    int precs[2];
    return n >= 2 ? (uint64_t)(n - 1) * sampler_precs(mode, precs) : 0;
}

// Enqueues one batch of the Clifford & Clifford loop on c->stream (eagerly or
// into a stream capture): init, then for k = 1..n plan / scan / walk /
// reduce (k >= 2) and draw, then the occupation counts.  Kernels read their
// arguments from `da` (device); `a` gives launch shapes.  *kernels counts
// the kernels enqueued.
int enqueue_sampler_batch(bs_ctx* c, const bs::CcArgs& a, const bs::CcArgs* da, bs_mode mode, uint64_t* kernels) {
    unsigned long long* ctl = static_cast<unsigned long long*>(c->ctl.p);
    int rc;
    cudaError_t e = bs::launch_cc_init(a, da, c->stream);
    if (e != cudaSuccess) return fail(BS_ECUDA, "sampler init: %s", cudaGetErrorString(e));
    ++*kernels;
    for (int k = 1; k <= a.n; ++k) {
        if (k >= 2) {
            if ((e = bs::launch_cc_plan(a, da, k, c->stream)) != cudaSuccess)
                return fail(BS_ECUDA, "sampler plan: %s", cudaGetErrorString(e));
            if ((e = bs::launch_cc_scan(a, da, k, c->stream)) != cudaSuccess)
                return fail(BS_ECUDA, "sampler scan: %s", cudaGetErrorString(e));
            *kernels += 2;
            int precs[2];
            const int np = sampler_precs(mode, precs);
            for (int pi = 0; pi < np; ++pi) {
                const int prec = precs[pi];
                bs::WalkArgs w;
                std::memset(&w, 0, sizeof(w));
                w.jobs = a.jobs;
                w.njobs = a.S;
                w.job_list = a.lists + prec * a.S;
                w.njobs_dev = a.list_len + prec;
                w.data = a.data;
                w.meta = a.meta;
                w.partials = a.partials;
                w.total_tasks = 0;
                w.total_dev = a.total + prec;
                w.counter = a.counter + prec;
                w.status = reinterpret_cast<int*>(ctl + kCtlStatus);
                w.deadline_rel_ns = c->deadline_s > 0 ? (unsigned long long)(c->deadline_s * 1e9) : 0ull;
                w.max_K = k;
                if ((rc = launch_walk(c, w, prec, BS_KIND_MINORS))) return rc;
                c->stats.kernel_launches--;  // the caller counts every kernel
                ++*kernels;
            }
            if ((e = bs::launch_reduce(a.jobs, a.S, a.partials, a.meta, a.minors, nullptr, k, c->stream)) !=
                cudaSuccess)
                return fail(BS_ECUDA, "sampler reduce: %s", cudaGetErrorString(e));
            ++*kernels;
        }
        if ((e = bs::launch_cc_draw(a, da, k, c->stream)) != cudaSuccess)
            return fail(BS_ECUDA, "sampler draw: %s", cudaGetErrorString(e));
        ++*kernels;
    }
    if ((e = bs::launch_cc_counts(a, da, c->stream)) != cudaSuccess)
        return fail(BS_ECUDA, "sampler counts: %s", cudaGetErrorString(e));
    ++*kernels;
    return BS_OK;
}

int sample_dev(bs_ctx* c, const double2* dU, int m_rows, int m_cols, int ld, const int* occ, int n_samples,
               uint64_t seed, int m_det, bs_mode mode, int* dout, int* dtrace = nullptr) {
    if (m_rows <= 0 || m_cols <= 0) return fail(BS_EINVAL, "bad interferometer size %d x %d", m_rows, m_cols);
    if (ld < m_cols) return fail(BS_EINVAL, "leading dimension %d < columns %d", ld, m_cols);
    if (m_rows > 8192) return fail(BS_EINVAL, "at most 8192 output modes are supported");
    if (!occ) return fail(BS_EINVAL, "input occupation is NULL");
    if (n_samples < 0) return fail(BS_EINVAL, "negative sample count");
    if (m_det <= 0 || m_det > m_rows) m_det = m_rows;
    std::vector<int> inputs;
    for (int i = 0; i < m_cols; ++i) {
        if (occ[i] < 0) return fail(BS_EINVAL, "negative occupation in mode %d", i);
        for (int t = 0; t < occ[i]; ++t) inputs.push_back(i);
    }
    const int n = (int)inputs.size();
    if (n > BS_MAX_N) return fail(BS_EINVAL, "n = %d photons exceeds the limit %d", n, BS_MAX_N);
    if (n_samples == 0) return BS_OK;
    if (n == 0) {
        BS_CUDA(cudaMemsetAsync(dout, 0, (size_t)n_samples * m_det * sizeof(int), c->stream));
        return BS_OK;
    }
    // worst-case tasks of one chain at the last step (C <= 2^(n-2)), over
    // the kernels a chain may be given (bs_choose_log2L gives at most
    // 2 x target tasks unless the chunk length is capped, and then at most
    // C / (cpt 2^log2max) + 1; cpt >= 16 for FP64 minors, 8 for FP32, 4 for DF)
    uint64_t cmax = n >= 2 ? (1ull << (n - 2)) : 1ull;
    uint64_t tasks_stride = 2 * BS_TARGET_TASKS_MANY + 1;
    {
        int precs[2];
        const int np = sampler_precs(mode, precs);
        for (int pi = 0; pi < np; ++pi) {
            const uint64_t cpt_min = precs[pi] == BS_PREC_FP64 ? 16 : precs[pi] == BS_PREC_FP32 ? 8 : 4;
            tasks_stride = std::max<uint64_t>(tasks_stride, cmax / (cpt_min << c->log2max[precs[pi]]) + 2);
        }
    }
    // a step-k job has <= k - 1 digit rows, K = k <= n columns, n' = k - 1;
    // a chain's data slot fits the widest row stride (DF: multiples of 8)
    const int64_t meta_stride = BS_META_SIZE(n, n, n), data_stride = (int64_t)n * BS_ROW_STRIDE_DF(n);
    // chains per pass: bounded by the budget (or 2 GiB of partials per pass)
    const size_t per_chain = (size_t)tasks_stride * n * sizeof(bs_zdd) + (size_t)data_stride * 16 +
                             meta_stride * 4 + sizeof(bs_job) + (size_t)n * (8 + 16) + 8 + 64;
    size_t cap_bytes = (size_t)2 << 30;
    if (c->budget) {
        size_t free_b = c->budget > c->used ? c->budget - c->used : 0;
        cap_bytes = std::min(cap_bytes, free_b / 2 + c->cc_partials.n);
    }
    int S_max = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_samples, cap_bytes / per_chain));
    int rc;
    const int S0 = std::min(S_max, n_samples);
    if ((rc = ensure(c, c->cc_inputs, n * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->cc_cols, (size_t)S0 * n * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->cc_rows, (size_t)S0 * n * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->cc_jobs, (size_t)S0 * sizeof(bs_job)))) return rc;
    if ((rc = ensure(c, c->cc_meta, (size_t)S0 * meta_stride * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->cc_data, (size_t)S0 * data_stride * 16))) return rc;
    if ((rc = ensure(c, c->cc_lists, (size_t)S0 * BS_NPREC * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->cc_partials, (size_t)S0 * tasks_stride * n * sizeof(bs_zdd)))) return rc;
    if ((rc = ensure(c, c->cc_minors, (size_t)S0 * n * sizeof(double2)))) return rc;
    if ((rc = ensure(c, c->ctl, kCtlSlots * 8))) return rc;
    int* h = static_cast<int*>(stage(c, n * sizeof(int)));
    if (!h) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    std::memcpy(h, inputs.data(), n * sizeof(int));
    BS_CUDA(cudaMemcpyAsync(c->cc_inputs.p, h, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaEventRecord(c->stage_ev[c->stage_cur], c->stream));
    // counters, totals and status; the statistics slots are cleared only by
    // bs_ctx_reset_stats
    BS_CUDA(cudaMemsetAsync(c->ctl.p, 0, kCtlStats * 8, c->stream));
    BS_CUDA(cudaMemsetAsync(static_cast<unsigned long long*>(c->ctl.p) + kCtlListLen, 0, (kCtlSlots - kCtlListLen) * 8, c->stream));
    unsigned long long* ctl = static_cast<unsigned long long*>(c->ctl.p);
    if ((rc = ensure(c, c->cc_args, sizeof(bs::CcArgs)))) return rc;
    bs::CcArgs* da = static_cast<bs::CcArgs*>(c->cc_args.p);
    for (int base = 0; base < n_samples; base += S_max) {
        bs::CcArgs a;
        std::memset(&a, 0, sizeof(a));
        a.S = std::min(S_max, n_samples - base);
        a.n = n;
        a.m_rows = m_rows;
        a.m_det = m_det;
        a.ld = ld;
        a.seed = seed;
        a.sample_base = (uint64_t)base;
        a.U = dU;
        a.inputs = static_cast<const int*>(c->cc_inputs.p);
        a.cols = static_cast<int*>(c->cc_cols.p);
        a.rows = static_cast<int*>(c->cc_rows.p);
        a.jobs = static_cast<bs_job*>(c->cc_jobs.p);
        a.meta = static_cast<int*>(c->cc_meta.p);
        a.data = c->cc_data.p;
        a.partials = static_cast<bs_zdd*>(c->cc_partials.p);
        a.minors = static_cast<double2*>(c->cc_minors.p);
        a.total = ctl + kCtlTotal;
        a.counter = ctl + kCtlCounter;
        a.stats = ctl + kCtlStats;
        a.lists = static_cast<int*>(c->cc_lists.p);
        a.list_len = reinterpret_cast<int*>(ctl + kCtlListLen);
        a.out = dout + (size_t)base * m_det;
        a.trace = dtrace ? dtrace + (size_t)base * n : nullptr;
        a.meta_stride = meta_stride;
        a.data_stride = data_stride;
        a.tasks_stride = (int64_t)tasks_stride;
        a.mode = (int)mode;
        a.log2max64 = c->log2max[BS_PREC_FP64];
        a.log2max32 = c->log2max[BS_PREC_FP32];
        a.log2maxdf = c->log2max[BS_PREC_DF];
        a.mixed_log2_tol = c->mixed_log2_tol;
        a.mixed_fallback = kMixedFallback;
        // the kernels read the arguments from device memory (pageable copy:
        // staged before cudaMemcpyAsync returns, so `a` may go out of scope)
        BS_CUDA(cudaMemcpyAsync(da, &a, sizeof(a), cudaMemcpyHostToDevice, c->stream));
        // eager launches when graphs are off, on the legacy default stream
        // (it cannot be captured), and when the caller is already capturing
        // this stream (the caller's graph then records these launches); with
        // profiling on, the graph carries the walk timing events
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (c->stream != nullptr) BS_CUDA(cudaStreamIsCapturing(c->stream, &cap));
        if (!c->use_graphs || c->stream == nullptr || c->stream == cudaStreamPerThread ||
            cap != cudaStreamCaptureStatusNone) {
            uint64_t kernels = 0;
            if ((rc = enqueue_sampler_batch(c, a, da, mode, &kernels))) return rc;
            c->stats.kernel_launches += kernels;
            continue;
        }
        // replay the captured step loop while shapes and buffers are unchanged
        const uint64_t dl = c->deadline_s > 0 ? (uint64_t)(c->deadline_s * 1e9) : 0;
        std::vector<uint64_t> key = {(uint64_t)a.S, (uint64_t)n, (uint64_t)m_rows, (uint64_t)m_det, (uint64_t)ld,
                                     (uint64_t)a.mode, (uint64_t)a.log2max64, (uint64_t)a.log2max32,
                                     (uint64_t)a.log2maxdf,
                                     (uint64_t)(uintptr_t)dU, (uint64_t)(uintptr_t)c->cc_cols.p,
                                     (uint64_t)(uintptr_t)c->cc_rows.p, (uint64_t)(uintptr_t)c->cc_jobs.p,
                                     (uint64_t)(uintptr_t)c->cc_meta.p, (uint64_t)(uintptr_t)c->cc_data.p,
                                     (uint64_t)(uintptr_t)c->cc_partials.p, (uint64_t)(uintptr_t)c->cc_minors.p,
                                     (uint64_t)(uintptr_t)c->cc_lists.p, (uint64_t)(uintptr_t)c->ctl.p,
                                     (uint64_t)(uintptr_t)da, tasks_stride, dl, (uint64_t)(uintptr_t)c->stream,
                                     (uint64_t)c->profiling};
        // (the MIXED threshold is read by the device planner from *da, so a
        // replay follows a changed threshold without a new capture)
        harvest_graph_timing(c);
        if (!c->cc_exec || key != c->cc_key) {
            if (c->cc_exec) {
                cudaGraphExecDestroy(c->cc_exec);
                c->cc_exec = nullptr;
            }
            drop_graph_timing(c);
            // with profiling on, the walk timing events are captured as
            // event-record nodes: they move from the eager list to the graph
            const size_t timed_before = c->timed.size();
            BS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            uint64_t kernels = 0;
            const uint64_t walks_before = c->stats.walk_launches;
            rc = enqueue_sampler_batch(c, a, da, mode, &kernels);
            c->stats.walk_launches = walks_before;  // counted per replay below
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            c->cc_graph_timed.assign(c->timed.begin() + timed_before, c->timed.end());
            c->timed.resize(timed_before);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                drop_graph_timing(c);
                return rc;
            }
            if (e != cudaSuccess) return fail(BS_ECUDA, "sampler graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&c->cc_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->cc_exec = nullptr;
                return fail(BS_ECUDA, "sampler graph instantiate: %s", cudaGetErrorString(e));
            }
            c->cc_key = key;
            c->cc_graph_kernels = kernels;
        }
        BS_CUDA(cudaGraphLaunch(c->cc_exec, c->stream));
        c->cc_timing_pending = !c->cc_graph_timed.empty();
        c->stats.kernel_launches += c->cc_graph_kernels;
        c->stats.walk_launches += kernels_walks(n, mode);
    }
    return BS_OK;
}

uint64_t read_device_stat(bs_ctx* c, int which) {
    if (!c->ctl.p) return 0;
    unsigned long long v = 0;
    cudaMemcpy(&v, static_cast<unsigned long long*>(c->ctl.p) + kCtlStats + which, 8, cudaMemcpyDeviceToHost);
    return v;
}

}  // namespace

// ====================================================================== C ABI
#pragma GCC visibility push(default)
extern "C" {

int bs_ctx_create(bs_ctx** out, int device, size_t mem_budget_bytes) {
    if (!out) return fail(BS_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count <= 0) {
        cudaGetLastError();
        return fail(BS_ENODEV, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    if (device < 0 || device >= count) return fail(BS_EINVAL, "device %d out of range [0, %d)", device, count);
    bs_ctx* c = new bs_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        e = cudaEventCreateWithFlags(&c->stage_ev[b], cudaEventDisableTiming);
    c->stream = c->own;
    if (e != cudaSuccess) {
        cudaGetLastError();
        bs_ctx_destroy(c);  // releases whatever was created
        return fail(BS_ECUDA, "context setup: %s", cudaGetErrorString(e));
    }
    // control words (task counters, status, statistics) start at zero
    if (ensure(c, c->ctl, kCtlSlots * 8) != BS_OK || cudaMemset(c->ctl.p, 0, kCtlSlots * 8) != cudaSuccess) {
        cudaGetLastError();
        bs_ctx_destroy(c);
        return fail(BS_ENOMEM, "could not allocate the control block");
    }
    *out = c;
    return BS_OK;
}

void bs_ctx_destroy(bs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& t : c->timed) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    DevBuf* bufs[] = {&c->src,       &c->jobs,     &c->meta,     &c->data64,  &c->data32,      &c->partials,
                      &c->out,       &c->out_lo,   &c->ctl,      &c->cc_inputs, &c->cc_cols,   &c->cc_rows,
                      &c->cc_jobs,   &c->cc_meta,  &c->cc_data,  &c->cc_partials, &c->cc_minors, &c->cc_out,
                      &c->cc_U, &c->cc_lists, &c->cc_args};
    if (c->cc_exec) cudaGraphExecDestroy(c->cc_exec);
    drop_graph_timing(c);
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    for (DevBuf* b : bufs) release(c, *b);
    for (int b = 0; b < 2; ++b)
        if (c->h_stage[b]) cudaFreeHost(c->h_stage[b]);
    if (c->h_back) cudaFreeHost(c->h_back);
    for (int b = 0; b < 2; ++b)
        if (c->stage_ev[b]) cudaEventDestroy(c->stage_ev[b]);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

const char* bs_last_error(const bs_ctx*) { return bs::last_error(); }

int bs_ctx_set_stream(bs_ctx* c, void* stream) {
    if (!ok_ctx(c)) return BS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->stream = static_cast<cudaStream_t>(stream);
    return BS_OK;
}

int bs_ctx_use_own_stream(bs_ctx* c) {
    if (!ok_ctx(c)) return BS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->stream = c->own;
    return BS_OK;
}

int bs_ctx_sync(bs_ctx* c) {
    if (!ok_ctx(c)) return BS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return sync_and_check(c);
}

int bs_ctx_set_deadline(bs_ctx* c, double seconds) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!(seconds >= 0.0)) return fail(BS_EINVAL, "deadline must be >= 0");
    c->deadline_s = seconds;
    return BS_OK;
}

int bs_ctx_set_chunk_log2(bs_ctx* c, bs_mode mode, int log2_chunk_max) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode");
    if (log2_chunk_max < 4 || log2_chunk_max > 20) return fail(BS_EINVAL, "log2 chunk %d outside [4, 20]", log2_chunk_max);
    c->log2max[mode] = log2_chunk_max;
    return BS_OK;
}

int bs_ctx_set_mixed_tolerance(bs_ctx* c, double tol) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!(tol > 0.0)) return fail(BS_EINVAL, "MIXED tolerance must be positive");
    std::lock_guard<std::mutex> lk(c->mu);
    c->mixed_log2_tol = tol >= 1e300 ? 1e30f : (float)std::log2(tol);
    return BS_OK;
}

int bs_ctx_get_chunk_log2(const bs_ctx* c, bs_mode mode) {
    if (!c || !valid_mode(mode)) return BS_EINVAL;
    return c->log2max[mode];
}

int bs_perm(bs_ctx* c, const bs_c128* A, int rows, int cols, int ld, const int* row_mult, const int* col_mult,
            bs_mode mode, bs_c128* out, bs_c128* out_lo) {
    if (!out) return fail(BS_EINVAL, "out is NULL");
    IntPlan p;
    std::vector<double2> hi, lo;
    int rc = single_job(c, A, rows, cols, ld, row_mult, col_mult, BS_KIND_PERM, mode, p, hi, lo);
    if (rc) return rc;
    out->re = hi[0].x;
    out->im = hi[0].y;
    if (out_lo) {
        out_lo->re = lo[0].x;
        out_lo->im = lo[0].y;
    }
    return BS_OK;
}

int bs_perm_formula(bs_ctx* c, const bs_c128* A, int n, int ld, bs_formula formula, bs_c128* out, bs_c128* out_lo) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!out) return fail(BS_EINVAL, "out is NULL");
    if (n < 0 || n > BS_MAX_N) return fail(BS_EINVAL, "matrix size %d outside [0, %d]", n, BS_MAX_N);
    IntPlan p;
    int rc;
    if (formula == BS_FORMULA_BBFG) {
        int ones[BS_MAX_N];
        for (int i = 0; i < n; ++i) ones[i] = 1;
        rc = plan_job(n, n, ones, ones, BS_KIND_PERM, p);
    } else if (formula == BS_FORMULA_RYSER || formula == BS_FORMULA_NW) {
        rc = plan_formula(n, formula == BS_FORMULA_RYSER ? BS_JOB_RYSER : BS_JOB_NW, p);
    } else {
        return fail(BS_EINVAL, "unknown formula %d", (int)formula);
    }
    if (rc) return rc;
    std::vector<double2> hi, lo;
    rc = run_single(c, A, n, n, ld, BS_KIND_PERM, BS_FP64, p, hi, lo);
    if (rc) return rc;
    out->re = hi[0].x;
    out->im = hi[0].y;
    if (out_lo) {
        out_lo->re = lo[0].x;
        out_lo->im = lo[0].y;
    }
    return BS_OK;
}

int bs_laplace_minors(bs_ctx* c, const bs_c128* A, int rows, int cols, int ld, const int* row_mult,
                      const int* col_mult, bs_mode mode, bs_c128* minors) {
    if (!minors) return fail(BS_EINVAL, "minors is NULL");
    IntPlan p;
    std::vector<double2> hi, lo;
    int rc = single_job(c, A, rows, cols, ld, row_mult, col_mult, BS_KIND_MINORS, mode, p, hi, lo);
    if (rc) return rc;
    for (int j = 0; j < cols; ++j) {
        const int e = p.trivial ? (col_mult[j] > 0 ? 0 : -1) : first_product_col(col_mult, j);
        if (e < 0) {
            minors[j].re = 0.0;
            minors[j].im = 0.0;
        } else {
            minors[j].re = hi[e].x;
            minors[j].im = hi[e].y;
        }
    }
    return BS_OK;
}

static int batch_common(bs_ctx* c, int count, const bs_c128* A_packed, const int64_t* a_offset, const int* rows,
                        const int* cols, const int* mult_packed, const int64_t* row_mult_off,
                        const int64_t* col_mult_off, bs_mode mode, std::vector<IntPlan>& plans) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (count < 0) return fail(BS_EINVAL, "negative count");
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (count > 0 && (!a_offset || !rows || !cols || !mult_packed || !row_mult_off || !col_mult_off))
        return fail(BS_EINVAL, "NULL batch array");
    plans.resize(count);
    for (int b = 0; b < count; ++b) {
        int rc = plan_job(rows[b], cols[b], mult_packed + row_mult_off[b], mult_packed + col_mult_off[b],
                          BS_KIND_PERM, plans[b]);
        if (rc) return fail(rc, "item %d: %s", b, std::string(bs::last_error()).c_str());
        if (!plans[b].trivial && (!A_packed || a_offset[b] < 0))
            return fail(BS_EINVAL, "item %d: bad matrix pointer or offset", b);
    }
    return BS_OK;
}

// Identity of a batch for graph replay: everything the plan and the device
// sequence depend on except the device pointers (compared separately).
static std::vector<int64_t> batch_key(const bs_ctx* c, int count, const int64_t* a_offset, const int* rows,
                                      const int* cols, const int* mult_packed, const int64_t* row_mult_off,
                                      const int64_t* col_mult_off, bs_mode mode) {
    std::vector<int64_t> k;
    int64_t dl = 0;
    std::memcpy(&dl, &c->deadline_s, sizeof(dl));
    k.insert(k.end(), {(int64_t)count, (int64_t)mode, (int64_t)c->log2max[0], (int64_t)c->log2max[1],
                       (int64_t)c->log2max[2], dl, tol_key(c)});
    for (int b = 0; b < count; ++b) {
        k.insert(k.end(), {a_offset[b], (int64_t)rows[b], (int64_t)cols[b]});
        for (int r = 0; r < rows[b]; ++r) k.push_back(mult_packed[row_mult_off[b] + r]);
        for (int j = 0; j < cols[b]; ++j) k.push_back(mult_packed[col_mult_off[b] + j]);
    }
    return k;
}

int bs_perm_batch(bs_ctx* c, int count, const bs_c128* A_packed, const int64_t* a_offset, const int* rows,
                  const int* cols, const int* mult_packed, const int64_t* row_mult_off, const int64_t* col_mult_off,
                  bs_mode mode, bs_c128* out) {
    std::vector<IntPlan> plans;
    int rc = batch_common(c, count, A_packed, a_offset, rows, cols, mult_packed, row_mult_off, col_mult_off, mode,
                          plans);
    if (rc) return rc;
    if (count == 0) return BS_OK;
    if (!out) return fail(BS_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    BS_CUDA(cudaSetDevice(c->device));
    size_t total = 0;
    std::vector<int64_t> off(count);
    for (int b = 0; b < count; ++b) {
        off[b] = (int64_t)total;
        if (!plans[b].trivial) total += (size_t)rows[b] * cols[b];
    }
    if ((rc = ensure(c, c->src, total * sizeof(bs_c128)))) return rc;
    if ((rc = ensure(c, c->out, count * sizeof(double2)))) return rc;
    bs_c128* h = static_cast<bs_c128*>(stage(c, total * sizeof(bs_c128)));
    if (!h) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    for (int b = 0; b < count; ++b)
        if (!plans[b].trivial) copy_matrix(h + off[b], A_packed + a_offset[b], rows[b], cols[b], cols[b]);
    BS_CUDA(cudaMemcpyAsync(c->src.p, h, total * sizeof(bs_c128), cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaEventRecord(c->stage_ev[c->stage_cur], c->stream));
    // the staged sources are contiguous: the key uses their offsets
    const std::vector<int64_t> key =
        batch_key(c, count, off.data(), rows, cols, mult_packed, row_mult_off, col_mult_off, mode);
    rc = batch_walk(c, plans, key, off.data(), cols, static_cast<const double2*>(c->src.p),
                    static_cast<double2*>(c->out.p), mode, nullptr);
    if (rc) return rc;
    std::vector<double2> res(count);
    BS_CUDA(cudaMemcpyAsync(res.data(), c->out.p, count * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = sync_and_check(c))) return rc;
    for (int b = 0; b < count; ++b) {
        if (plans[b].trivial) {
            out[b].re = 1.0;
            out[b].im = 0.0;
        } else {
            out[b].re = res[b].x;
            out[b].im = res[b].y;
        }
    }
    return BS_OK;
}

int bs_perm_batch_dev(bs_ctx* c, int count, const bs_c128* A_packed_dev, const int64_t* a_offset, const int* rows,
                      const int* cols, const int* mult_packed, const int64_t* row_mult_off,
                      const int64_t* col_mult_off, bs_mode mode, bs_c128* out_dev) {
    std::vector<IntPlan> plans;
    int rc = batch_common(c, count, A_packed_dev, a_offset, rows, cols, mult_packed, row_mult_off, col_mult_off,
                          mode, plans);
    if (rc) return rc;
    if (count == 0) return BS_OK;
    if (!out_dev) return fail(BS_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    BS_CUDA(cudaSetDevice(c->device));
    std::vector<int> trivial;
    for (int b = 0; b < count; ++b)
        if (plans[b].trivial) trivial.push_back(b);
    const std::vector<int64_t> key =
        batch_key(c, count, a_offset, rows, cols, mult_packed, row_mult_off, col_mult_off, mode);
    rc = batch_walk(c, plans, key, a_offset, cols, reinterpret_cast<const double2*>(A_packed_dev),
                    reinterpret_cast<double2*>(out_dev), mode, nullptr);
    if (rc) return rc;
    if (!trivial.empty()) {
        static const double2 one = {1.0, 0.0};
        for (int b : trivial)
            BS_CUDA(cudaMemcpyAsync(out_dev + b, &one, sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    }
    return BS_OK;
}

int bs_sample_dev(bs_ctx* c, const bs_c128* U_dev, int m_rows, int m_cols, int ld, const int* input_occupation,
                  int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out_dev) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (!U_dev || (!out_dev && n_samples > 0)) return fail(BS_EINVAL, "NULL device pointer");
    std::lock_guard<std::mutex> lk(c->mu);
    BS_CUDA(cudaSetDevice(c->device));
    return sample_dev(c, reinterpret_cast<const double2*>(U_dev), m_rows, m_cols, ld, input_occupation, n_samples,
                      seed, m_detected, mode, out_dev);
}

// Host-memory sampling: U up, counts (and, when rows_out is given, the drawn
// rows of every step) back.
static int sample_host(bs_ctx* c, const bs_c128* U, int m_rows, int m_cols, int ld, const int* input_occupation,
                       int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out, int* rows_out) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (!U || (!out && n_samples > 0)) return fail(BS_EINVAL, "NULL pointer");
    if (m_rows <= 0 || m_cols <= 0 || ld < m_cols) return fail(BS_EINVAL, "bad interferometer size");
    if (n_samples <= 0) return n_samples < 0 ? fail(BS_EINVAL, "negative sample count") : BS_OK;
    if (!input_occupation) return fail(BS_EINVAL, "input occupation is NULL");
    int n = 0;
    for (int i = 0; i < m_cols; ++i) n += input_occupation[i] > 0 ? input_occupation[i] : 0;
    const int mdet = (m_detected <= 0 || m_detected > m_rows) ? m_rows : m_detected;
    std::lock_guard<std::mutex> lk(c->mu);
    BS_CUDA(cudaSetDevice(c->device));
    const size_t ub = (size_t)m_rows * m_cols * sizeof(bs_c128);
    const size_t ob = (size_t)n_samples * mdet * sizeof(int);
    const size_t tb = rows_out ? (size_t)n_samples * n * sizeof(int) : 0;
    int rc;
    if ((rc = ensure(c, c->cc_U, ub))) return rc;
    if ((rc = ensure(c, c->cc_out, ob + tb))) return rc;
    bs_c128* h = static_cast<bs_c128*>(stage(c, std::max(ub, ob + tb)));
    if (!h) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    copy_matrix(h, U, m_rows, m_cols, ld);
    BS_CUDA(cudaMemcpyAsync(c->cc_U.p, h, ub, cudaMemcpyHostToDevice, c->stream));
    BS_CUDA(cudaEventRecord(c->stage_ev[c->stage_cur], c->stream));
    int* d_out = static_cast<int*>(c->cc_out.p);
    int* d_trace = rows_out ? d_out + (size_t)n_samples * mdet : nullptr;
    rc = sample_dev(c, static_cast<const double2*>(c->cc_U.p), m_rows, m_cols, m_cols, input_occupation, n_samples,
                    seed, mdet, mode, d_out, d_trace);
    if (rc) return rc;
    // read back through a staging buffer (stage() waits until no copy out of
    // it is pending)
    void* hb = stage(c, ob + tb);
    if (!hb) return fail(BS_ENOMEM, "pinned host staging allocation failed");
    BS_CUDA(cudaMemcpyAsync(hb, c->cc_out.p, ob + tb, cudaMemcpyDeviceToHost, c->stream));
    if ((rc = sync_and_check(c))) return rc;
    std::memcpy(out, hb, ob);
    if (rows_out) std::memcpy(rows_out, static_cast<char*>(hb) + ob, tb);
    return BS_OK;
}

int bs_sample_ex(bs_ctx* c, const bs_c128* U, int m_rows, int m_cols, int ld, const int* input_occupation,
                 int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out) {
    return sample_host(c, U, m_rows, m_cols, ld, input_occupation, n_samples, seed, m_detected, mode, out, nullptr);
}

int bs_sample_trace(bs_ctx* c, const bs_c128* U, int m_rows, int m_cols, int ld, const int* input_occupation,
                    int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out, int* rows_out) {
    if (!rows_out && n_samples > 0) return fail(BS_EINVAL, "rows_out is NULL");
    return sample_host(c, U, m_rows, m_cols, ld, input_occupation, n_samples, seed, m_detected, mode, out, rows_out);
}

int bs_sample(bs_ctx* c, const bs_c128* U, int m, const int* input_occupation, int n_samples, uint64_t seed,
              bs_mode mode, int* out) {
    return bs_sample_ex(c, U, m, m, m, input_occupation, n_samples, seed, m, mode, out);
}

int bs_ctx_set_graphs(bs_ctx* c, int on) {
    if (!ok_ctx(c)) return BS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->use_graphs = on != 0;
    return BS_OK;
}

int bs_ctx_set_profiling(bs_ctx* c, int on) {
    if (!ok_ctx(c)) return BS_EINVAL;
    c->profiling = on != 0;
    return BS_OK;
}

// Converts recorded walk event pairs into durations (stream must be idle).
static void collect_timed(bs_ctx* c) {
    harvest_graph_timing(c);
    for (auto& t : c->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
            c->stats.walk_ms[t.prec] += ms;
            c->stats.timed_launches[t.prec]++;
            c->walk_log.push_back(ms);
        } else {
            cudaGetLastError();
        }
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    c->timed.clear();
}

int bs_ctx_get_walk_times(bs_ctx* c, double* ms_out, int max_entries) {
    if (!ok_ctx(c) || (max_entries > 0 && !ms_out)) return fail(BS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(BS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    collect_timed(c);
    int n = (int)c->walk_log.size();
    for (int i = 0; i < n && i < max_entries; ++i) ms_out[i] = c->walk_log[i];
    c->walk_log.clear();
    return n;
}

int bs_ctx_get_stats(bs_ctx* c, bs_stats* out) {
    if (!ok_ctx(c) || !out) return fail(BS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(BS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    collect_timed(c);
    *out = c->stats;
    for (int p = 0; p < BS_NPREC; ++p) {
        out->addends[p] += read_device_stat(c, 2 * p);
        out->addend_flops[p] += read_device_stat(c, 2 * p + 1);
    }
    return BS_OK;
}

int bs_ctx_reset_stats(bs_ctx* c) {
    if (!ok_ctx(c)) return BS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& t : c->timed) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    c->timed.clear();
    c->cc_timing_pending = false;
    c->walk_log.clear();
    c->stats = bs_stats();
    if (c->ctl.p) cudaMemset(static_cast<unsigned long long*>(c->ctl.p) + kCtlStats, 0, 2 * BS_NPREC * 8);
    return BS_OK;
}

int bs_measure_fma_rates(bs_ctx* c, double* fp64, double* fp32) {
    if (!ok_ctx(c) || !fp64 || !fp32) return fail(BS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaError_t e = bs::measure_fma_rates(c->device, fp64, fp32);
    if (e != cudaSuccess) return fail(BS_ECUDA, "microbenchmark: %s", cudaGetErrorString(e));
    return BS_OK;
}

int bs_tune(bs_ctx* c, bs_mode mode, int kind, int K, int* best_log2, double* best_addends_per_s) {
    if (!ok_ctx(c)) return BS_EINVAL;
    if (!valid_mode(mode)) return fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (kind != 0 && kind != 1) return fail(BS_EINVAL, "kind must be 0 (permanent) or 1 (minors)");
    if (K < 4 || K > BS_MAX_COLS) return fail(BS_EINVAL, "K must be in [4, %d]", BS_MAX_COLS);
    // synthetic problem: K product columns, up to 25 distinct rows (at most
    // 2^24 addends), the remaining photons on the first rows (multiplicity 2)
    const int n = kind == 0 ? K : K - 1;
    const int R = std::min(n, 25);
    std::vector<bs_c128> A((size_t)R * K);
    uint64_t x = 0x9E3779B97F4A7C15ull ^ (uint64_t)K;
    for (auto& z : A) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        z.re = ((double)(x >> 11) * 0x1.0p-53 - 0.5) / std::sqrt((double)K);
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        z.im = ((double)(x >> 11) * 0x1.0p-53 - 0.5) / std::sqrt((double)K);
    }
    std::vector<int> M(R, 1), N(K, 1);
    for (int extra = n - R, r = 0; extra > 0; --extra, ++r) M[r % R] += 1;
    const int saved = c->log2max[mode];
    const bool prof = c->profiling;
    c->profiling = true;
    double best_ms = 1e300;
    int best = saved;
    uint64_t C = 0;
    for (int cand = 8; cand <= 14; cand += 2) {
        c->log2max[mode] = cand;
        IntPlan p;
        std::vector<double2> hi, lo;
        double ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            std::vector<double> times;
            int rc = single_job(c, A.data(), R, K, K, M.data(), N.data(), kind == 0 ? BS_KIND_PERM : BS_KIND_MINORS,
                                mode, p, hi, lo);
            if (rc) {
                c->log2max[mode] = saved;
                c->profiling = prof;
                return rc;
            }
            double t = 0;
            for (auto& e : c->timed) {
                float f = 0.f;
                cudaEventElapsedTime(&f, e.e0, e.e1);
                t += f;
                cudaEventDestroy(e.e0);
                cudaEventDestroy(e.e1);
            }
            c->timed.clear();
            if (rep == 1) ms = t;
        }
        C = p.C;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    c->log2max[mode] = best;
    c->profiling = prof;
    if (best_log2) *best_log2 = best;
    if (best_addends_per_s) *best_addends_per_s = (double)C / (best_ms * 1e-3);
    return BS_OK;
}

int bs_debug_gray_walk(int ndigits, int nbin, const int* radix, uint64_t start, int steps, int* deltas, int* moved,
                       uint64_t* weights) {
    if (ndigits < 0 || ndigits > BS_MAX_DIGITS || nbin < 0 || nbin > ndigits || !radix || steps < 0)
        return fail(BS_EINVAL, "bad digit description");
    uint64_t C = 1;
    for (int j = 0; j < ndigits; ++j) {
        if (radix[j] < 2 || radix[j] > 61 || (j < nbin && radix[j] != 2))
            return fail(BS_EINVAL, "bad radix %d at digit %d", radix[j], j);
        C *= (uint64_t)radix[j];
        if (C > (1ull << 50)) return fail(BS_EINVAL, "too many addends");
    }
    if (start >= C || start + (uint64_t)steps > C) return fail(BS_EINVAL, "walk leaves [0, C)");
    // the same per-job binomial table the kernels read
    uint64_t binom[BS_MAX_DIGITS * 62];
    int at = 0;
    for (int j = 0; j < ndigits; ++j)
        for (int d = 0; d < radix[j]; ++d) binom[at++] = bs_binom(radix[j] - 1, d);
    bs_gray g;
    bs_gray_decode(g, start, nbin, ndigits, radix, binom);
    for (int s = 0; s < steps; ++s) {
        if (s > 0) {
            int coef, wch;
            int row = bs_gray_step(g, radix, &coef, &wch, binom);
            if (moved) moved[s] = row;
        } else if (moved) {
            moved[0] = -1;
        }
        if (deltas)
            for (int j = 0; j < ndigits; ++j) deltas[(size_t)s * ndigits + j] = bs_gray_delta(g, j);
        if (weights) weights[s] = g.w;
    }
    return BS_OK;
}

int bs_debug_mixed_error(int rows, int cols, const int* row_mult, const int* col_mult, int kind, int chunk_log2,
                         double* log2_err, int* log2L, int* plan) {
    if (!log2_err) return fail(BS_EINVAL, "log2_err is NULL");
    IntPlan p;
    int rc = plan_job(rows, cols, row_mult, col_mult, kind == 1 ? BS_KIND_MINORS : BS_KIND_PERM, p);
    if (rc) return rc;
    if (p.trivial) {
        *log2_err = -1000.0;
        if (log2L) *log2L = 0;
        if (plan) *plan = 1;
        return BS_OK;
    }
    const int l32 = chunk_log2 > 0
                        ? chunk_log2
                        : bs_choose_log2L_single(p.C, bs_chunks_per_task(p.kind, 1, p.K), bs_default_log2max(BS_PREC_FP32),
                                                 BS_TARGET_TASKS_SINGLE_FP32);
    std::vector<double> q_work(BS_MIXED_QMAX + 1);
    *log2_err = bs_mixed_log2_error(p.radix, p.nrows, p.pinned_m, p.K, p.n, l32, q_work.data());
    if (log2L) *log2L = l32;
    if (plan)
        *plan = bs_mixed_fp32_plan(p.radix, p.nrows, p.pinned_m, p.K, p.n, l32, BS_MIXED_LOG2_TOL_DEFAULT,
                                   q_work.data());
    return BS_OK;
}

int bs_debug_plan(int rows, int cols, const int* row_mult, const int* col_mult, int kind, int64_t* info) {
    if (!info) return fail(BS_EINVAL, "info is NULL");
    IntPlan p;
    int rc = plan_job(rows, cols, row_mult, col_mult, kind == 1 ? BS_KIND_MINORS : BS_KIND_PERM, p);
    if (rc) return rc;
    info[0] = p.trivial ? 0 : (int64_t)p.C;
    info[1] = p.nrows;
    info[2] = p.nbin;
    info[3] = p.K;
    info[4] = p.trans ? 1 : 0;
    info[5] = p.pinned_src;
    // chunking of this job planned alone in FP64 mode (default maximum 2^12)
    const int kd = kind == 1 ? BS_KIND_MINORS : BS_KIND_PERM;
    const int cpt = bs_chunks_per_task(kd, 0, p.K);
    const int l = p.trivial ? 0 : bs_choose_log2L_single(p.C, cpt, bs_default_log2max(BS_PREC_FP64), BS_TARGET_TASKS_SINGLE);
    const uint64_t per = (uint64_t)cpt << l;
    info[6] = l;
    info[7] = p.trivial ? 0 : (int64_t)((p.C + per - 1) / per);
    return BS_OK;
}

}  // extern "C"
#pragma GCC visibility pop
