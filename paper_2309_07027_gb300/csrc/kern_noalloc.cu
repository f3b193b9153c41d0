// Allocation-free permanent: bs_perm_noalloc.
//
// Who needs it: callers that must not allocate device memory at the moment
// they ask for a permanent -- hosts whose memory manager owns a fixed device
// budget and forbids allocations outside it (a cudaMalloc there can fail or
// take memory the manager has promised elsewhere), and real-time loops that
// may not enter the CUDA allocator (cudaMalloc and cudaFree can synchronise
// the device and have no latency bound).  bs_perm (a context with grow-only
// buffers) allocates on first use and whenever a larger problem arrives;
// this entry point never does.  It has no deadline: the walk runs to the
// end of the job.
//
// How: every byte of device scratch (job descriptor, metadata, the compacted
// matrix, the packed column data, the per-task partial sums, the result and
// the control words) lives in one file-scope __device__ array of
// BS_NOALLOC_SCRATCH_BYTES = 8 MiB.  Every GPU that loads the library keeps
// that array until the process exits.  Host staging uses the caller's stack.
// The kernels are the same pack / walk / reduce kernels bs_perm uses.
//
// In host code the array's name is only a host-side handle, not a device
// address: the first call on each device (with that device current) asks the
// runtime for the array's device address with cudaGetSymbolAddress, checks
// the result and caches it; kernels only ever receive that address.
//
// All calls share the one array and leave their data in it; the counter and
// status words are cleared on every call.  Calls whose work overlaps on the
// GPU (different host threads, or different streams without ordering) race on
// the array and give wrong results; serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bs.h"
#include "bs_job.h"
#include "kernels.h"
#include "plan.h"
#include "sample.h"

#define BS_NOALLOC_SCRATCH_BYTES (8u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[BS_NOALLOC_SCRATCH_BYTES];

namespace {

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t kCtl = 0;                                        // u64 counter, int status at +8
constexpr size_t kJob = 256;                                      // one bs_job
constexpr size_t kMeta = 512;                                     // <= BS_META_SIZE(48, 48, 48) ints
constexpr size_t kOut = 2304;                                     // result hi / lo (2 x 16 bytes)
constexpr size_t kSrc = 2560;                                     // compacted matrix, <= 48 x 48
constexpr size_t kData = kSrc + (size_t)BS_MAX_N * BS_MAX_N * 16;  // packed c0 / 2a
constexpr size_t kPart = kData + (size_t)(1 + BS_MAX_N) * BS_ROW_STRIDE_DF(BS_MAX_N) * 16;
constexpr size_t kPartSlots = (BS_NOALLOC_SCRATCH_BYTES - kPart) / sizeof(bs_zdd);
// Chunk-length cap of this call's planner: 2^12 in every mode (the task
// count of a job falls with the cap, and this one sets the size limit the
// header states); only jobs beyond about 2^31 addends reach it.
constexpr int kLog2Max = 12;
static_assert(kPart % 256 == 0 && kData % 256 == 0, "scratch regions must stay aligned");
static_assert(kMeta + BS_META_SIZE(BS_MAX_DIGITS, BS_MAX_COLS, BS_MAX_N) * 4 <= kOut, "metadata region too small");

std::mutex g_setup_mu;
unsigned char* g_scratch_dev[64];  // device address of the array, per device

int scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return bs::fail(BS_EINVAL, "device %d out of range for the scratch table", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return bs::fail(BS_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                            cudaGetErrorString(e));
        }
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return BS_OK;
}

#define NA_CUDA(call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return bs::fail(BS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

}  // namespace

#pragma GCC visibility push(default)
extern "C" int bs_perm_noalloc(const bs_c128* A, int rows, int cols, int ld, const int* row_mult,
                               const int* col_mult, bs_mode mode, void* stream, bs_c128* out, bs_c128* out_lo) {
    if (!out) return bs::fail(BS_EINVAL, "out is NULL");
    if (mode != BS_FP64 && mode != BS_MIXED && mode != BS_DF64) return bs::fail(BS_EINVAL, "unknown mode %d", (int)mode);
    if (rows < 0 || cols < 0) return bs::fail(BS_EINVAL, "negative matrix size %d x %d", rows, cols);
    if ((rows > 0 && !row_mult) || (cols > 0 && !col_mult)) return bs::fail(BS_EINVAL, "multiplicity array is NULL");
    // compact away zero multiplicities (at most BS_MAX_N rows / columns remain)
    int rsrc[BS_MAX_N], csrc[BS_MAX_N], Mc[BS_MAX_N], Nc[BS_MAX_N];
    int nr = 0, nc = 0;
    for (int r = 0; r < rows; ++r) {
        if (row_mult[r] < 0) return bs::fail(BS_EINVAL, "row multiplicity of row %d is negative", r);
        if (row_mult[r] == 0) continue;
        if (nr == BS_MAX_N) return bs::fail(BS_EINVAL, "n exceeds the limit %d", BS_MAX_N);
        rsrc[nr] = r;
        Mc[nr++] = row_mult[r];
    }
    for (int j = 0; j < cols; ++j) {
        if (col_mult[j] < 0) return bs::fail(BS_EINVAL, "column multiplicity of column %d is negative", j);
        if (col_mult[j] == 0) continue;
        if (nc == BS_MAX_N) return bs::fail(BS_EINVAL, "n exceeds the limit %d", BS_MAX_N);
        csrc[nc] = j;
        Nc[nc++] = col_mult[j];
    }
    bs::IntPlan p;
    int rc = bs::plan_job(nr, nc, Mc, Nc, BS_KIND_PERM, p);
    if (rc) return rc;
    if (p.trivial) {
        out->re = 1.0;
        out->im = 0.0;
        if (out_lo) out_lo->re = out_lo->im = 0.0;
        return BS_OK;
    }
    if (!A) return bs::fail(BS_EINVAL, "matrix pointer is NULL");
    if (ld < cols) return bs::fail(BS_EINVAL, "leading dimension %d < columns %d", ld, cols);
    int prec = mode == BS_DF64 ? BS_PREC_DF : BS_PREC_FP64;
    int reseed = 0;
    if (mode == BS_MIXED) {
        double q_work[BS_MIXED_QMAX + 1];  // the rule's scratch, on the stack
        const int l32 = bs_choose_log2L_single(p.C, bs_chunks_per_task(BS_KIND_PERM, BS_PREC_FP32, p.K), kLog2Max,
                                               BS_TARGET_TASKS_SINGLE_FP32);
        const int plan = bs_mixed_fp32_plan(p.radix, p.nrows, p.pinned_m, p.K, p.n, l32, BS_MIXED_LOG2_TOL_DEFAULT,
                                            q_work);
        prec = plan ? BS_PREC_FP32 : BS_MIXED_FALLBACK_PREC;
        reseed = plan == 2 ? BS_FP32_RESEED_LOG2 : 0;
    }
    const int cpt = bs_chunks_per_task(BS_KIND_PERM, prec, p.K);
    const int log2L = bs_choose_log2L_single(p.C, cpt, kLog2Max,
                                             prec == BS_PREC_FP32 ? BS_TARGET_TASKS_SINGLE_FP32 : BS_TARGET_TASKS_SINGLE);
    const uint64_t per = (uint64_t)cpt << log2L;
    const uint64_t ntasks = (p.C + per - 1) / per;
    if (ntasks > kPartSlots)
        return bs::fail(BS_EINVAL,
                        "bs_perm_noalloc: %llu addends need %llu task slots; its fixed scratch holds %zu "
                        "(about %.3g addends); use bs_perm",
                        (unsigned long long)p.C, (unsigned long long)ntasks, kPartSlots,
                        (double)kPartSlots * (double)per);
    // host-side descriptors on the stack
    bs_c128 Ac[BS_MAX_N * BS_MAX_N];
    for (int r = 0; r < nr; ++r)
        for (int j = 0; j < nc; ++j) Ac[r * nc + j] = A[(size_t)rsrc[r] * ld + csrc[j]];
    bs_job jb;
    std::memset(&jb, 0, sizeof(jb));
    jb.C = p.C;
    jb.ntasks = (uint32_t)ntasks;
    jb.K = p.K;
    jb.nrows = p.nrows;
    jb.nbin = p.nbin;
    jb.kind = BS_KIND_PERM;
    jb.log2L = log2L;
    jb.n = p.n;
    jb.normalize = prec != BS_PREC_FP64 ? 1 : 0;
    jb.prec = prec;
    jb.reseed_log2 = reseed;
    jb.src_ld = nc;
    jb.src_trans = p.trans ? 1 : 0;
    int meta[BS_META_SIZE(BS_MAX_DIGITS, BS_MAX_COLS, BS_MAX_N)];
    int m = 0;
    for (int d = 0; d < p.nrows; ++d) meta[m++] = p.radix[d];
    for (int d = 0; d < p.nrows; ++d) meta[m++] = p.digit_src[d];
    for (int j = 0; j < p.K; ++j) meta[m++] = p.col_src[j];
    for (int j = 0; j < p.K; ++j) meta[m++] = 0;
    meta[m++] = p.pinned_src;
    meta[m++] = 0;                                            // pad; the binomial table follows
    for (int t = 0; t < 2 * (p.nrows + p.n); ++t) meta[m++] = 0;
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    unsigned char* scr = nullptr;
    if ((rc = scratch_address(dev, &scr))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NA_CUDA(cudaMemsetAsync(scr + kCtl, 0, 16, s));
    NA_CUDA(cudaMemcpyAsync(scr + kJob, &jb, sizeof(jb), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(scr + kMeta, meta, (size_t)m * sizeof(int), cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(scr + kSrc, Ac, (size_t)nr * nc * sizeof(bs_c128), cudaMemcpyHostToDevice, s));
    const bs_job* djob = reinterpret_cast<const bs_job*>(scr + kJob);
    int* dmeta = reinterpret_cast<int*>(scr + kMeta);
    NA_CUDA(bs::launch_pack(djob, 1, reinterpret_cast<const double2*>(scr + kSrc), dmeta, scr + kData, prec, s));
    bs::WalkArgs w;
    std::memset(&w, 0, sizeof(w));
    w.jobs = djob;
    w.njobs = 1;
    w.data = scr + kData;
    w.meta = dmeta;
    w.partials = reinterpret_cast<bs_zdd*>(scr + kPart);
    w.total_tasks = ntasks;
    w.counter = reinterpret_cast<unsigned long long*>(scr + kCtl);
    w.status = reinterpret_cast<int*>(scr + kCtl + 8);
    w.max_K = p.K;
    NA_CUDA(prec == BS_PREC_DF     ? bs::launch_walk_df_perm(w, s)
            : prec == BS_PREC_FP32 ? bs::launch_walk_fp32_perm(w, s)
                                   : bs::launch_walk_fp64_perm(w, s));
    NA_CUDA(bs::launch_reduce(djob, 1, w.partials, dmeta, reinterpret_cast<double2*>(scr + kOut),
                              reinterpret_cast<double2*>(scr + kOut + 16), 1, s));
    double2 res[2];
    int status = 0;
    NA_CUDA(cudaMemcpyAsync(res, scr + kOut, sizeof(res), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaMemcpyAsync(&status, scr + kCtl + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (status != BS_STATUS_OK) return bs::fail(BS_ECUDA, "walk kernel status %d", status);
    out->re = res[0].x;
    out->im = res[0].y;
    if (out_lo) {
        out_lo->re = res[1].x;
        out_lo->im = res[1].y;
    }
    return BS_OK;
}
#pragma GCC visibility pop
