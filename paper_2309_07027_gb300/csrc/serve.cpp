// Serving engine: continuous batching of permanent, minors and sampling
// requests from many concurrent clients.  A sampling request is a whole
// Clifford & Clifford chain (Sec. 4): its interferometer, permuted inputs
// and drawn rows stay resident on the device, and each step's minors job
// joins the shared walk launches of the next tick while the draw of the next
// row and the planning of the next job run on the device (chain_advance).
//
// A scheduler thread runs ticks.  Each tick
//   1. admits waiting requests in arrival order while a slot is free and the
//      request's device memory (matrix, packed columns, task partials,
//      results) fits the budget (first-fit arena inside one device block);
//      newly admitted jobs are packed on the device;
//   2. walks a slice of every resident job's tasks: the tick's task budget
//      is shared equally among resident jobs, so a short request admitted
//      while long ones are running finishes within a tick or two instead of
//      waiting for them (iteration-level scheduling);
//   3. reduces the jobs whose last task ran, copies their results back and
//      releases their memory and slot.
// All tasks of one tick run in one persistent walk launch per (precision,
// kind, column bucket).  A job's chunking depends only on the job, partials
// are indexed by the job's own task number and summed in a fixed order, so a
// result is bit-identical whether it ran alone or mixed with others.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "bs.h"
#include "bs_job.h"
#include "kernels.h"
#include "plan.h"
#include "sample.h"

namespace {

using clock_type = std::chrono::steady_clock;
constexpr size_t kAlign = 256;
// chunk-length caps (by precision) of served jobs: a context's defaults, so
// that a served sample plans every step as bs_sample does

// First-fit allocator over [0, size) with coalescing free ranges.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
        used_ = 0;
        peak_ = 0;
    }
    // returns offset or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                peak_ = std::max(peak_.load(), used_.load());
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    // the engine thread alone allocates and releases (a tick's descriptors
    // outside the lock); the counters are read by bs_server_get_stats
    std::atomic<size_t> used_{0}, peak_{0};
};

struct Request {
    int64_t id = 0;
    int kind = BS_KIND_PERM;
    bs::IntPlan plan;
    int cols = 0;                      // caller's column count (minors output)
    std::vector<int> col_mult;         // caller's column multiplicities (minors mapping)
    std::vector<bs_c128> mat;          // caller's rows x cols, copied with ld = cols
    int rows = 0;
    clock_type::time_point t_submit, t_done;
    // device placement (byte offsets into the arena)
    size_t off = 0, bytes = 0;
    int64_t src_off = 0, data_off = 0, meta_off = 0, part_off = 0;
    int slot = -1;                     // result slot (BS_MAX_COLS values)
    int prec = BS_PREC_FP64, cpt = 32, log2L = 6, ncols = 1, reseed = 0;
    uint32_t ntasks = 0, done = 0;
    int status = 0;                    // 0 pending, 1 done, <0 error code
    std::vector<bs_c128> result;
    bool cancel = false;               // set by bs_server_cancel; released between ticks
    // sampling chains: one Clifford & Clifford sample
    bool chain = false;
    int k = 0;                         // step whose row is drawn next (1 = first)
    bool chain_done = false;
    int m_rows = 0, m_cols = 0, m_det = 0, n = 0;
    uint64_t seed = 0, sample = 0;
    std::vector<int> inputs;           // expanded input columns
    std::vector<int> counts;           // result: m_det occupation counts
    bs_job job_host{};                 // the pending step's job, as planned on the device
    uint64_t tasks_stride = 0;         // task partial slots per step
    // byte offsets of the chain's regions inside its arena block
    size_t c_u = 0, c_in = 0, c_cols = 0, c_rows = 0, c_cnt = 0, c_job = 0, c_meta = 0, c_data = 0, c_part = 0;
};

}  // namespace

struct bs_server {
    int device = 0;
    bs_mode mode = BS_FP64;
    int max_active = 64;
    int tick_tasks = 8192;
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    void* arena_base = nullptr;
    Arena arena;
    void* h_pinned = nullptr;
    size_t h_pinned_n = 0;
    void* d_ctl = nullptr;  // counters (64) + status
    void* d_out = nullptr;  // max_active result slots of BS_MAX_COLS complex values
    std::vector<int> free_slots;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> waiting;
    std::vector<Request*> active;
    std::map<int64_t, Request*> all;
    int64_t next_id = 0;
    bool stop = false;
    std::thread engine;
    std::string fatal;

    // statistics
    uint64_t submitted = 0, completed = 0, ticks = 0, walk_launches = 0, cancelled = 0;
    double busy_s = 0;
    int max_resident = 0;
    std::vector<double> latencies_ms;
};

namespace {

int ensure_pinned(bs_server* s, size_t bytes) {
    if (s->h_pinned_n >= bytes) return BS_OK;
    if (s->h_pinned) cudaFreeHost(s->h_pinned);
    s->h_pinned = nullptr;
    size_t want = std::max(bytes, s->h_pinned_n * 2);
    if (cudaHostAlloc(&s->h_pinned, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        s->h_pinned_n = 0;
        return bs::fail(BS_ENOMEM, "pinned staging allocation failed");
    }
    s->h_pinned_n = want;
    return BS_OK;
}

// Lays out a chain's regions (byte offsets from the start of its block) and
// returns the block size: U, inputs, permuted columns, drawn rows, counts,
// the job descriptor, metadata, packed data (widest row stride) and task
// partials for its largest step.
size_t chain_layout(Request& r) {
    auto up = [](size_t b) { return (b + kAlign - 1) / kAlign * kAlign; };
    size_t at = 0;
    auto take = [&](size_t b) {
        const size_t o = at;
        at += up(std::max<size_t>(b, 1));
        return o;
    };
    r.c_u = take((size_t)r.m_rows * r.m_cols * 16);
    r.c_in = take((size_t)r.n * 4);
    r.c_cols = take((size_t)r.n * 4);
    r.c_rows = take((size_t)r.n * 4);
    r.c_cnt = take((size_t)r.m_det * 4);
    r.c_job = take(sizeof(bs_job));
    r.c_meta = take((size_t)BS_META_SIZE(r.n, r.n, r.n) * 4);
    r.c_data = take((size_t)r.n * BS_ROW_STRIDE_DF(r.n) * 16);
    r.c_part = take((size_t)r.tasks_stride * r.n * sizeof(bs_zdd));
    return at;
}

// Bytes a request needs on the device.
size_t request_bytes(const Request& r) {
    const bs::IntPlan& p = r.plan;
    auto up = [](size_t b) { return (b + kAlign - 1) / kAlign * kAlign; };
    size_t b = 0;
    b += up((size_t)r.rows * r.cols * 16);                          // source matrix
    b += up((size_t)(1 + p.nrows) * BS_ROW_STRIDE_P(p.K, r.prec) * 16);  // packed c0 / 2a
    b += up((size_t)BS_META_SIZE(p.nrows, p.K, p.n) * 4);                // metadata
    b += up((size_t)r.ntasks * r.ncols * sizeof(bs_zdd));            // task partials
    return b;
}

void finish(bs_server* s, Request* r, int status) {
    r->status = status;
    r->t_done = clock_type::now();
    if (status == 1) {
        s->completed++;
        s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    } else if (status == BS_ECANCELED) {
        s->cancelled++;
    }
}

// One scheduling tick; called by the engine thread with the lock released.
// `admit` are requests already given arena space.
int run_tick(bs_server* s, std::vector<Request*>& admit, std::vector<Request*>& resident) {
    char* base = static_cast<char*>(s->arena_base);
    // 1. upload and pack the admitted jobs
    std::vector<bs_job> packjobs[BS_NPREC];
    for (Request* r : admit) {
        if (r->chain) {  // U and the input columns; the chain's kernels start it (below)
            cudaError_t e = cudaMemcpyAsync(base + r->off + r->c_u, r->mat.data(), r->mat.size() * 16,
                                            cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(base + r->off + r->c_in, r->inputs.data(), r->inputs.size() * 4,
                                    cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return bs::fail(BS_ECUDA, "server upload: %s", cudaGetErrorString(e));
            continue;
        }
        const bs::IntPlan& p = r->plan;
        size_t at = r->off;
        auto take = [&](size_t b) {
            size_t o = at;
            at += (b + kAlign - 1) / kAlign * kAlign;
            return o;
        };
        const size_t src_b = take((size_t)r->rows * r->cols * 16);
        const size_t data_b = take((size_t)(1 + p.nrows) * BS_ROW_STRIDE_P(p.K, r->prec) * 16);
        const size_t meta_b = take((size_t)BS_META_SIZE(p.nrows, p.K, p.n) * 4);
        const size_t part_b = take((size_t)r->ntasks * r->ncols * sizeof(bs_zdd));
        r->src_off = (int64_t)(src_b / 16);
        r->data_off = (int64_t)(data_b / (r->prec == BS_PREC_FP32 ? 8 : 16));
        r->meta_off = (int64_t)(meta_b / 4);
        r->part_off = (int64_t)(part_b / sizeof(bs_zdd));
        int meta[BS_META_SIZE(BS_MAX_DIGITS, BS_MAX_COLS, BS_MAX_N)];
        int m = 0;
        for (int d = 0; d < p.nrows; ++d) meta[m++] = p.radix[d];
        for (int d = 0; d < p.nrows; ++d) meta[m++] = p.digit_src[d];
        for (int j = 0; j < p.K; ++j) meta[m++] = p.col_src[j];
        for (int j = 0; j < p.K; ++j) meta[m++] = 0;
        meta[m++] = p.pinned_src;
        meta[m++] = 0;                                        // pad; the binomial table follows
        for (int t = 0; t < 2 * (p.nrows + p.n); ++t) meta[m++] = 0;
        cudaError_t e = cudaMemcpyAsync(base + src_b, r->mat.data(), r->mat.size() * 16, cudaMemcpyHostToDevice,
                                        s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + meta_b, meta, (size_t)m * 4, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return bs::fail(BS_ECUDA, "server upload: %s", cudaGetErrorString(e));
        bs_job jb;
        std::memset(&jb, 0, sizeof(jb));
        jb.C = p.C;
        jb.ntasks = r->ntasks;
        jb.K = p.K;
        jb.nrows = p.nrows;
        jb.nbin = p.nbin;
        jb.kind = r->kind;
        jb.log2L = r->log2L;
        jb.n = p.n;
        jb.normalize = r->prec != BS_PREC_FP64 ? 1 : 0;
        jb.prec = r->prec;
        jb.reseed_log2 = r->reseed;
        jb.data_off = r->data_off;
        jb.meta_off = r->meta_off;
        jb.partial_off = r->part_off;
        jb.out_index = r->slot * BS_MAX_COLS;
        jb.src_off = r->src_off;
        jb.src_ld = r->cols;
        jb.src_trans = p.trans ? 1 : 0;
        packjobs[r->prec].push_back(jb);
    }
    // 2. this tick's slices: equal share of the task budget per resident job
    std::vector<bs_job> walk;
    std::vector<Request*> walk_req;
    size_t walking = 0;
    for (Request* r : resident) walking += r->done < r->ntasks ? 1 : 0;
    const uint32_t share = std::max<uint32_t>(1, (uint32_t)(s->tick_tasks / std::max<size_t>(1, walking)));
    for (Request* r : resident) {
        if (r->done >= r->ntasks) continue;  // a chain between steps, or a newly admitted chain
        bs_job jb;
        if (r->chain) {
            jb = r->job_host;
        } else {
            const bs::IntPlan& p = r->plan;
            std::memset(&jb, 0, sizeof(jb));
            jb.C = p.C;
            jb.K = p.K;
            jb.nrows = p.nrows;
            jb.nbin = p.nbin;
            jb.kind = r->kind;
            jb.log2L = r->log2L;
            jb.n = p.n;
            jb.prec = r->prec;
            jb.reseed_log2 = r->reseed;
            jb.data_off = r->data_off;
            jb.meta_off = r->meta_off;
            jb.partial_off = r->part_off;
        }
        jb.ntasks = std::min(share, r->ntasks - r->done);
        jb.task_offset = r->done;
        walk.push_back(jb);
        walk_req.push_back(r);
    }
    // sort into kernel groups, largest slices first
    std::vector<size_t> order(walk.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    // kernel bucket of a job: 4-column buckets, 8-column for double-float
    auto bucket = [](const bs_job& j) { return j.prec == BS_PREC_DF ? (j.K + 7) / 8 : (j.K + 3) / 4; };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const bs_job &x = walk[a], &y = walk[b];
        if (x.prec != y.prec) return x.prec < y.prec;
        if (x.kind != y.kind) return x.kind < y.kind;
        if (bucket(x) != bucket(y)) return bucket(x) < bucket(y);
        return x.ntasks > y.ntasks;
    });
    std::vector<bs_job> tick;
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < order.size();) {
        size_t j = i;
        const bs_job& g0 = walk[order[i]];
        uint64_t tb = 0;
        const size_t gstart = tick.size();
        while (j < order.size() && walk[order[j]].prec == g0.prec && walk[order[j]].kind == g0.kind &&
               bucket(walk[order[j]]) == bucket(g0)) {
            bs_job jb = walk[order[j]];
            jb.task_begin = tb;
            tb += jb.ntasks;
            tick.push_back(jb);
            ++j;
        }
        groups.push_back({gstart, tick.size()});
        i = j;
    }
    // finishing jobs reduce over all their tasks
    std::vector<bs_job> fin;
    std::vector<Request*> fin_req;
    for (size_t i = 0; i < walk.size(); ++i) {
        Request* r = walk_req[i];
        if (r->done + walk[i].ntasks == r->ntasks) {
            bs_job jb = walk[i];
            jb.ntasks = r->ntasks;
            jb.task_offset = 0;
            jb.out_index = r->slot * BS_MAX_COLS;
            fin.push_back(jb);
            fin_req.push_back(r);
        }
    }
    // chains that draw a row this tick: the admitted ones (step 1) first,
    // then those whose step job finishes now
    std::vector<Request*> adv;
    int n_init = 0, max_m_rows = 1;
    for (Request* r : admit)
        if (r->chain) adv.push_back(r);
    n_init = (int)adv.size();
    for (Request* r : fin_req)
        if (r->chain) adv.push_back(r);
    std::vector<bs::ChainDesc> descs;
    size_t back_bytes = 0;
    for (Request* r : adv) {
        char* cb = base + r->off;
        bs::ChainDesc d;
        std::memset(&d, 0, sizeof(d));
        d.U = reinterpret_cast<const double2*>(cb + r->c_u);
        d.m_rows = r->m_rows;
        d.m_cols = r->m_cols;
        d.m_det = r->m_det;
        d.n = r->n;
        d.seed = r->seed;
        d.sample = r->sample;
        d.inputs = reinterpret_cast<const int*>(cb + r->c_in);
        d.cols = reinterpret_cast<int*>(cb + r->c_cols);
        d.rows = reinterpret_cast<int*>(cb + r->c_rows);
        d.counts = reinterpret_cast<int*>(cb + r->c_cnt);
        d.job = reinterpret_cast<bs_job*>(cb + r->c_job);
        d.meta_off = (int64_t)((r->off + r->c_meta) / 4);
        d.data_byte_off = (int64_t)(r->off + r->c_data);
        d.partial_off = (int64_t)((r->off + r->c_part) / sizeof(bs_zdd));
        d.out_index = r->slot * BS_MAX_COLS;
        d.k = r->k;
        d.rule.mode = (int)s->mode;
        d.rule.mixed_log2_tol = BS_MIXED_LOG2_TOL_DEFAULT;
        d.rule.mixed_fallback = BS_MIXED_FALLBACK_PREC;
        for (int q = 0; q < BS_NPREC; ++q) d.rule.log2max[q] = bs_default_log2max(q);
        descs.push_back(d);
        max_m_rows = std::max(max_m_rows, r->m_rows);
        back_bytes += r->k < r->n ? sizeof(bs_job) : (size_t)r->m_det * 4;
    }
    size_t npack = 0;
    for (int q = 0; q < BS_NPREC; ++q) npack += packjobs[q].size();
    const size_t nb_pack = npack * sizeof(bs_job);
    const size_t nb_tick = tick.size() * sizeof(bs_job), nb_fin = fin.size() * sizeof(bs_job);
    const size_t nb_chain = descs.size() * sizeof(bs::ChainDesc);
    size_t out_bytes = 0;
    for (Request* r : fin_req)
        if (!r->chain) out_bytes += (size_t)r->ncols * 16;
    int rc = ensure_pinned(s, nb_pack + nb_tick + nb_fin + nb_chain + out_bytes + back_bytes + 64);
    if (rc) return rc;
    // descriptors go to the tail of the arena's control block
    char* hp = static_cast<char*>(s->h_pinned);
    {
        size_t at = 0;
        for (int q = 0; q < BS_NPREC; ++q) {
            std::memcpy(hp + at, packjobs[q].data(), packjobs[q].size() * sizeof(bs_job));
            at += packjobs[q].size() * sizeof(bs_job);
        }
    }
    std::memcpy(hp + nb_pack, tick.data(), nb_tick);
    std::memcpy(hp + nb_pack + nb_tick, fin.data(), nb_fin);
    std::memcpy(hp + nb_pack + nb_tick + nb_fin, descs.data(), nb_chain);
    const size_t desc_bytes = nb_pack + nb_tick + nb_fin + nb_chain;
    size_t desc_off = s->arena.alloc(std::max<size_t>(desc_bytes, 16));
    if (desc_off == SIZE_MAX) return bs::fail(BS_ENOMEM, "server: no arena space for tick descriptors");
    cudaError_t e = cudaMemcpyAsync(base + desc_off, hp, desc_bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return bs::fail(BS_ECUDA, "server descriptors: %s", cudaGetErrorString(e));
    const bs_job* d_pack = reinterpret_cast<const bs_job*>(base + desc_off);
    const bs_job* d_tick = reinterpret_cast<const bs_job*>(base + desc_off + nb_pack);
    const bs_job* d_fin = reinterpret_cast<const bs_job*>(base + desc_off + nb_pack + nb_tick);
    const bs::ChainDesc* d_chain =
        reinterpret_cast<const bs::ChainDesc*>(base + desc_off + nb_pack + nb_tick + nb_fin);
    {
        size_t at = 0;
        for (int q = 0; q < BS_NPREC && e == cudaSuccess; ++q) {
            if (!packjobs[q].empty())
                e = bs::launch_pack(d_pack + at, (int)packjobs[q].size(), reinterpret_cast<const double2*>(base),
                                    reinterpret_cast<int*>(base), base, q, s->stream);
            at += packjobs[q].size();
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ctl, 0, 66 * 8, s->stream);
    unsigned long long* ctl = static_cast<unsigned long long*>(s->d_ctl);
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
        bs::WalkArgs w;
        std::memset(&w, 0, sizeof(w));
        w.jobs = d_tick + groups[gi].first;
        w.njobs = (int)(groups[gi].second - groups[gi].first);
        w.data = base;
        w.meta = reinterpret_cast<const int*>(base);
        w.partials = reinterpret_cast<bs_zdd*>(base);
        uint64_t tot = 0;
        int kmax = 0;
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            tot += tick[i].ntasks;
            kmax = std::max(kmax, tick[i].K);
        }
        w.total_tasks = tot;
        w.counter = ctl + gi;  // at most 2 x 2 x 12 + 2 x 6 = 60 groups
        w.status = reinterpret_cast<int*>(ctl + 64);
        w.max_K = kmax;
        const bs_job& g0 = tick[groups[gi].first];
        if (g0.prec == BS_PREC_DF)
            e = g0.kind == BS_KIND_PERM ? bs::launch_walk_df_perm(w, s->stream) : bs::launch_walk_df_minors(w, s->stream);
        else if (g0.prec == BS_PREC_FP32)
            e = g0.kind == BS_KIND_PERM ? bs::launch_walk_fp32_perm(w, s->stream) : bs::launch_walk_fp32_minors(w, s->stream);
        else
            e = g0.kind == BS_KIND_PERM ? bs::launch_walk_fp64_perm(w, s->stream) : bs::launch_walk_fp64_minors(w, s->stream);
        s->walk_launches++;
    }
    int maxc = 1;
    for (auto& jb : fin) maxc = std::max(maxc, jb.kind == BS_KIND_PERM ? 1 : jb.K);
    if (e == cudaSuccess && !fin.empty())
        e = bs::launch_reduce(d_fin, (int)fin.size(), reinterpret_cast<const bs_zdd*>(base),
                              reinterpret_cast<const int*>(base), static_cast<double2*>(s->d_out), nullptr, maxc,
                              s->stream);
    // chains: permute the admitted chains' inputs, then draw this tick's rows
    // and plan their next jobs (their step minors are in d_out)
    if (e == cudaSuccess && n_init > 0) e = bs::launch_chain_init(d_chain, n_init, s->stream);
    if (e == cudaSuccess && !descs.empty())
        e = bs::launch_chain_advance(d_chain, (int)descs.size(), max_m_rows, base,
                                     static_cast<const double2*>(s->d_out), s->stream);
    char* hout = hp + desc_bytes + 16;
    size_t at = 0;
    for (Request* r : fin_req) {
        if (e != cudaSuccess) break;
        if (r->chain) continue;
        e = cudaMemcpyAsync(hout + at, static_cast<double2*>(s->d_out) + (size_t)r->slot * BS_MAX_COLS,
                            (size_t)r->ncols * 16, cudaMemcpyDeviceToHost, s->stream);
        at += (size_t)r->ncols * 16;
    }
    char* hback = hout + at;
    size_t bat = 0;
    for (Request* r : adv) {
        if (e != cudaSuccess) break;
        if (r->k < r->n) {
            e = cudaMemcpyAsync(hback + bat, base + r->off + r->c_job, sizeof(bs_job), cudaMemcpyDeviceToHost,
                                s->stream);
            bat += sizeof(bs_job);
        } else {
            e = cudaMemcpyAsync(hback + bat, base + r->off + r->c_cnt, (size_t)r->m_det * 4, cudaMemcpyDeviceToHost,
                                s->stream);
            bat += (size_t)r->m_det * 4;
        }
    }
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp + desc_bytes, ctl + 64, 4, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    s->arena.release(desc_off, std::max<size_t>(desc_bytes, 16));
    if (e != cudaSuccess) return bs::fail(BS_ECUDA, "server tick: %s", cudaGetErrorString(e));
    std::memcpy(&status, hp + desc_bytes, 4);
    if (status != BS_STATUS_OK) return bs::fail(BS_ECUDA, "server walk status %d", status);
    for (size_t i = 0; i < walk.size(); ++i) walk_req[i]->done += walk[i].ntasks;
    bat = 0;
    for (Request* r : adv) {
        if (r->k < r->n) {
            std::memcpy(&r->job_host, hback + bat, sizeof(bs_job));
            bat += sizeof(bs_job);
            r->k += 1;  // the planned job is step k + 1's; its row is drawn when it completes
            r->ntasks = r->job_host.ntasks;
            r->done = 0;
            r->prec = r->job_host.prec;
        } else {
            r->counts.assign(reinterpret_cast<const int*>(hback + bat), reinterpret_cast<const int*>(hback + bat) + r->m_det);
            bat += (size_t)r->m_det * 4;
            r->chain_done = true;
        }
    }
    at = 0;
    for (Request* r : fin_req) {
        if (r->chain) continue;
        const double2* v = reinterpret_cast<const double2*>(hout + at);
        at += (size_t)r->ncols * 16;
        if (r->kind == BS_KIND_PERM) {
            r->result.assign(1, bs_c128{v[0].x, v[0].y});
        } else {
            r->result.assign(r->cols, bs_c128{0.0, 0.0});
            for (int j = 0; j < r->cols; ++j) {
                const int e2 = bs::first_product_col(r->col_mult.data(), j);
                if (e2 >= 0) r->result[j] = bs_c128{v[e2].x, v[e2].y};
            }
        }
    }
    return BS_OK;
}

void engine_loop(bs_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // admission: arrival order, slots and memory
        std::vector<Request*> admit;
        while (!s->waiting.empty() && (int)s->active.size() < s->max_active) {
            Request* r = s->waiting.front();
            size_t off = s->arena.alloc(r->bytes);
            if (off == SIZE_MAX) {
                if (s->active.empty()) {  // can never fit
                    s->waiting.pop_front();
                    finish(s, r, BS_ENOMEM);
                    s->cv_done.notify_all();
                    continue;
                }
                break;
            }
            r->off = off;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->waiting.pop_front();
            s->active.push_back(r);
            admit.push_back(r);
        }
        if (s->active.empty()) {
            s->cv_work.wait(lk, [&] { return s->stop || !s->waiting.empty(); });
            continue;
        }
        s->max_resident = std::max(s->max_resident, (int)s->active.size());
        std::vector<Request*> resident = s->active;
        lk.unlock();
        auto t0 = clock_type::now();
        int rc = run_tick(s, admit, resident);
        auto t1 = clock_type::now();
        lk.lock();
        s->busy_s += std::chrono::duration<double>(t1 - t0).count();
        s->ticks++;
        if (rc) {
            s->fatal = bs::last_error();
            for (Request* r : s->active) {
                s->arena.release(r->off, r->bytes);
                s->free_slots.push_back(r->slot);
                finish(s, r, rc);
            }
            s->active.clear();
            s->cv_done.notify_all();
            continue;
        }
        std::vector<Request*> still;
        for (Request* r : s->active) {
            const bool complete = r->chain ? r->chain_done : r->done == r->ntasks;
            if (complete || r->cancel) {
                // between ticks: no kernel of this request is in flight
                s->arena.release(r->off, r->bytes);
                s->free_slots.push_back(r->slot);
                finish(s, r, complete ? 1 : BS_ECANCELED);
            } else {
                still.push_back(r);
            }
        }
        s->active.swap(still);
        s->cv_done.notify_all();
    }
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

int bs_server_create(bs_server** out, int device, size_t mem_budget_bytes, int max_active, int tick_tasks,
                     bs_mode mode) {
    if (!out) return bs::fail(BS_EINVAL, "out is NULL");
    *out = nullptr;
    if (mode != BS_FP64 && mode != BS_MIXED && mode != BS_DF64) return bs::fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (max_active < 1 || tick_tasks < 1 || mem_budget_bytes < (64u << 10))
        return bs::fail(BS_EINVAL, "need max_active >= 1, tick_tasks >= 1, budget >= 64 KiB");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
        cudaGetLastError();
        return bs::fail(BS_ENODEV, "no CUDA device available");
    }
    if (device < 0 || device >= count) return bs::fail(BS_EINVAL, "device %d out of range", device);
    bs_server* s = new bs_server();
    s->device = device;
    s->mode = mode;
    s->max_active = max_active;
    s->tick_tasks = tick_tasks;
    s->budget = mem_budget_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, mem_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctl, 66 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_out, (size_t)max_active * BS_MAX_COLS * sizeof(double2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->arena_base) cudaFree(s->arena_base);
        if (s->d_ctl) cudaFree(s->d_ctl);
        if (s->d_out) cudaFree(s->d_out);
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return bs::fail(e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA, "server setup: %s",
                        cudaGetErrorString(e));
    }
    s->arena.reset(mem_budget_bytes);
    for (int i = max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->engine = std::thread(engine_loop, s);
    *out = s;
    return BS_OK;
}

void bs_server_destroy(bs_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->engine.joinable()) s->engine.join();
    for (auto& kv : s->all) delete kv.second;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->d_ctl) cudaFree(s->d_ctl);
    if (s->d_out) cudaFree(s->d_out);
    if (s->h_pinned) cudaFreeHost(s->h_pinned);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int64_t bs_server_submit(bs_server* s, int kind, const bs_c128* A, int rows, int cols, int ld, const int* row_mult,
                         const int* col_mult) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    if (kind != 0 && kind != 1) return bs::fail(BS_EINVAL, "kind must be 0 (permanent) or 1 (minors)");
    Request* r = new Request();
    r->kind = kind == 0 ? BS_KIND_PERM : BS_KIND_MINORS;
    int rc = bs::plan_job(rows, cols, row_mult, col_mult, r->kind, r->plan);
    if (rc) {
        delete r;
        return rc;
    }
    if (!r->plan.trivial && (!A || ld < cols)) {
        delete r;
        return bs::fail(BS_EINVAL, "bad matrix pointer or leading dimension");
    }
    r->rows = rows;
    r->cols = cols;
    r->col_mult.assign(col_mult, col_mult + cols);
    r->t_submit = clock_type::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->submitted++;
    if (r->plan.trivial) {
        r->result.assign(r->kind == BS_KIND_PERM ? 1 : cols, bs_c128{0.0, 0.0});
        if (r->kind == BS_KIND_PERM)
            r->result[0] = bs_c128{1.0, 0.0};
        else
            for (int j = 0; j < cols; ++j)
                if (col_mult[j] > 0) r->result[j] = bs_c128{1.0, 0.0};
        finish(s, r, 1);
        s->cv_done.notify_all();
        return r->id;
    }
    r->mat.resize((size_t)rows * cols);
    for (int i = 0; i < rows; ++i) std::memcpy(&r->mat[(size_t)i * cols], A + (size_t)i * ld, sizeof(bs_c128) * cols);
    r->prec = s->mode == BS_DF64 ? BS_PREC_DF : BS_PREC_FP64;
    if (s->mode == BS_MIXED) {
        double q_work[BS_MIXED_QMAX + 1];
        const int l32 = bs_choose_log2L(r->plan.C, bs_chunks_per_task(r->kind, BS_PREC_FP32, r->plan.K),
                                        BS_LOG2L_MIN_MANY, bs_default_log2max(BS_PREC_FP32), BS_TARGET_TASKS_MANY);
        const int plan = bs_mixed_fp32_plan(r->plan.radix, r->plan.nrows, r->plan.pinned_m, r->plan.K,
                                            r->plan.n, l32, BS_MIXED_LOG2_TOL_DEFAULT, q_work);
        r->prec = plan ? BS_PREC_FP32 : BS_MIXED_FALLBACK_PREC;
        r->reseed = plan == 2 ? BS_FP32_RESEED_LOG2 : 0;
    }
    r->cpt = bs_chunks_per_task(r->kind, r->prec, r->plan.K);
    r->log2L = bs_choose_log2L(r->plan.C, r->cpt, BS_LOG2L_MIN_MANY, bs_default_log2max(r->prec), BS_TARGET_TASKS_MANY);
    const uint64_t per = (uint64_t)r->cpt << r->log2L;
    r->ntasks = (uint32_t)((r->plan.C + per - 1) / per);
    r->ncols = r->kind == BS_KIND_PERM ? 1 : r->plan.K;
    r->bytes = request_bytes(*r);
    s->waiting.push_back(r);
    s->cv_work.notify_one();
    return r->id;
}

static int take_result(bs_server* s, Request* r, bs_c128* out, int out_len, double* latency_s) {
    int st = r->status;
    if (r->chain) return bs::fail(BS_EINVAL, "ticket %lld is a sampling request: use bs_server_wait_sample", (long long)r->id);
    if (st == 1) {
        const int need = (int)r->result.size();
        if (out_len < need) return bs::fail(BS_EINVAL, "output holds %d values, %d needed", out_len, need);
        if (out) std::memcpy(out, r->result.data(), sizeof(bs_c128) * need);
        if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    }
    s->all.erase(r->id);
    delete r;
    return st == 1 ? BS_OK
                   : bs::fail(st, "request %s", st == BS_ECANCELED ? "cancelled" : ("failed: " + s->fatal).c_str());
}

static int take_counts(bs_server* s, Request* r, int* counts, int len, double* latency_s) {
    int st = r->status;
    if (!r->chain) return bs::fail(BS_EINVAL, "ticket %lld is not a sampling request", (long long)r->id);
    if (st == 1) {
        if (len < r->m_det) return bs::fail(BS_EINVAL, "output holds %d counts, %d needed", len, r->m_det);
        if (counts) std::memcpy(counts, r->counts.data(), sizeof(int) * (size_t)r->m_det);
        if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    }
    s->all.erase(r->id);
    delete r;
    return st == 1 ? BS_OK
                   : bs::fail(st, "request %s", st == BS_ECANCELED ? "cancelled" : ("failed: " + s->fatal).c_str());
}

int bs_server_poll(bs_server* s, int64_t ticket, bs_c128* out, int out_len, double* latency_s) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return bs::fail(BS_EINVAL, "unknown ticket %lld", (long long)ticket);
    if (it->second->status == 0) return 0;
    int rc = take_result(s, it->second, out, out_len, latency_s);
    return rc == BS_OK ? 1 : rc;
}

int bs_server_wait(bs_server* s, int64_t ticket, bs_c128* out, int out_len, double* latency_s) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return bs::fail(BS_EINVAL, "unknown ticket %lld", (long long)ticket);
    Request* r = it->second;
    s->cv_done.wait(lk, [&] { return r->status != 0; });
    return take_result(s, r, out, out_len, latency_s);
}

int64_t bs_server_submit_sample(bs_server* s, const bs_c128* U, int m_rows, int m_cols, int ld,
                                const int* input_occupation, uint64_t seed, uint64_t sample, int m_detected) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    if (!U || !input_occupation) return bs::fail(BS_EINVAL, "NULL pointer");
    if (m_rows <= 0 || m_cols <= 0 || ld < m_cols) return bs::fail(BS_EINVAL, "bad interferometer size");
    if (m_rows > 8192) return bs::fail(BS_EINVAL, "at most 8192 output modes are supported");
    Request* r = new Request();
    r->chain = true;
    r->kind = BS_KIND_MINORS;
    for (int i = 0; i < m_cols; ++i) {
        if (input_occupation[i] < 0) {
            delete r;
            return bs::fail(BS_EINVAL, "negative occupation in mode %d", i);
        }
        for (int t = 0; t < input_occupation[i]; ++t) r->inputs.push_back(i);
    }
    r->n = (int)r->inputs.size();
    if (r->n > BS_MAX_N) {
        delete r;
        return bs::fail(BS_EINVAL, "n = %d photons exceeds the limit %d", r->n, BS_MAX_N);
    }
    r->m_rows = m_rows;
    r->m_cols = m_cols;
    r->m_det = (m_detected <= 0 || m_detected > m_rows) ? m_rows : m_detected;
    r->seed = seed;
    r->sample = sample;
    r->k = 1;
    r->rows = m_rows;
    r->cols = m_cols;
    r->ncols = r->n;
    r->t_submit = clock_type::now();
    if (r->n > 0) {
        r->mat.resize((size_t)m_rows * m_cols);
        for (int i = 0; i < m_rows; ++i)
            std::memcpy(&r->mat[(size_t)i * m_cols], U + (size_t)i * ld, sizeof(bs_c128) * m_cols);
        // task partial slots of the largest step (C <= 2^(n-2)) over the
        // kernels the mode may use (chunks per task >= 16 FP64, 8 FP32, 4 DF)
        const uint64_t cmax = r->n >= 2 ? (1ull << (r->n - 2)) : 1ull;
        uint64_t ts = 2 * BS_TARGET_TASKS_MANY + 1;
        const int precs_mixed[2] = {BS_PREC_FP32, BS_MIXED_FALLBACK_PREC};
        const int prec_one = s->mode == BS_DF64 ? BS_PREC_DF : BS_PREC_FP64;
        const int np = s->mode == BS_MIXED ? 2 : 1;
        for (int i = 0; i < np; ++i) {
            const int q = s->mode == BS_MIXED ? precs_mixed[i] : prec_one;
            const uint64_t cpt_min = q == BS_PREC_FP64 ? 16 : q == BS_PREC_FP32 ? 8 : 4;
            ts = std::max<uint64_t>(ts, cmax / (cpt_min << bs_default_log2max(q)) + 2);
        }
        r->tasks_stride = ts;
        r->bytes = chain_layout(*r);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->submitted++;
    if (r->n == 0) {  // no photons: the empty pattern
        r->counts.assign(r->m_det, 0);
        r->chain_done = true;
        finish(s, r, 1);
        s->cv_done.notify_all();
        return r->id;
    }
    s->waiting.push_back(r);
    s->cv_work.notify_one();
    return r->id;
}

int bs_server_poll_sample(bs_server* s, int64_t ticket, int* counts, int len, double* latency_s) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return bs::fail(BS_EINVAL, "unknown ticket %lld", (long long)ticket);
    if (it->second->status == 0) return 0;
    int rc = take_counts(s, it->second, counts, len, latency_s);
    return rc == BS_OK ? 1 : rc;
}

int bs_server_wait_sample(bs_server* s, int64_t ticket, int* counts, int len, double* latency_s) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return bs::fail(BS_EINVAL, "unknown ticket %lld", (long long)ticket);
    Request* r = it->second;
    s->cv_done.wait(lk, [&] { return r->status != 0; });
    return take_counts(s, r, counts, len, latency_s);
}

int bs_server_cancel(bs_server* s, int64_t ticket) {
    if (!s) return bs::fail(BS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return bs::fail(BS_EINVAL, "unknown ticket %lld", (long long)ticket);
    Request* r = it->second;
    if (r->status != 0) return bs::fail(BS_EINVAL, "ticket %lld has already finished", (long long)ticket);
    auto w = std::find(s->waiting.begin(), s->waiting.end(), r);
    if (w != s->waiting.end()) {  // not admitted: nothing on the device
        s->waiting.erase(w);
        finish(s, r, BS_ECANCELED);
        s->cv_done.notify_all();
        return BS_OK;
    }
    r->cancel = true;  // the engine releases it after the current tick
    return BS_OK;
}

int bs_server_get_stats(bs_server* s, bs_server_stats* out) {
    if (!s || !out) return bs::fail(BS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->ticks = s->ticks;
    out->walk_launches = s->walk_launches;
    out->busy_s = s->busy_s;
    out->max_resident = s->max_resident;
    out->mem_peak_bytes = s->arena.peak();
    out->mem_in_use_bytes = s->arena.used();
    out->resident = (int)s->active.size();
    out->waiting = (int)s->waiting.size();
    out->cancelled = s->cancelled;
    std::vector<double> l = s->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        out->p50_ms = l[(l.size() - 1) / 2];
        out->p99_ms = l[std::min(l.size() - 1, (size_t)(0.99 * (double)(l.size() - 1) + 0.5))];
        out->max_ms = l.back();
    }
    return BS_OK;
}

}  // extern "C"
#pragma GCC visibility pop
