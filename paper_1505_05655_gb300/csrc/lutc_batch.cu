// Batches: many independent rasters corrected together (lutc_batch_*).
//
// The paper's server takes tasks from many clients (Sections I-II).  A batch
// gathers such tasks -- images of uneven width, height, bit depth and band
// count, each with its own detector coefficients -- and runs them as one
// persistent TMA launch per phase: the launches walk the concatenation of
// every image's (band, strip, row) space, each block a contiguous run of
// about equal modelled cost (a strip row costs its valid columns plus one
// full strip's width).  Sequence per run:
//
//   reset (histograms, runs) -> pass 1 (stretch images of <= 12 bits) -> pass 1
//   (deeper ones: larger histograms, fewer blocks per SM) -> scan (one block
//   per image band) -> pass 2 (all stretch images) -> detector-only pass (all
//   uint16 images) -> images the TMA kernels cannot take, one by one
//
// The pass launches balance themselves at run time as well: each block claims
// its run a granule at a time and, once done, steals the upper half of the
// largest run left (lutc_tma.cu); the runs start from the planned boundaries,
// put back in place (with the histograms cleared) by one kernel at the start
// of every run.
//
// optionally captured once in a CUDA graph and replayed (lutc_batch_correct:
// planned, run once and released in one call).  All device data (job table,
// tensor maps, coefficient pointers, tables) lives in the caller's workspace:
// the library allocates no device memory here.
#include <cuda.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "lutc_internal.cuh"

using namespace lutc;

namespace {

enum Kind { kTmaStretch = 0, kTmaDetector = 1, kFallback = 2 };

// Pass 1 keeps a 2^bits x 4-byte histogram per block in shared memory: up to 12 bits it is small
// enough for 3 blocks per SM, above that only 2 fit.  Stretch jobs are therefore ordered
// small-table first and pass 1 runs as two launches, one per class.
constexpr int kSmallBits = 12;

// Each launch's blocks get contiguous runs of units (strip rows) of about equal cost.  A strip
// row's cost is modelled as its valid columns plus kRowOverhead: measured on GB300, a row of a
// narrow right-edge strip costs about as much as a full one (the tile's round trip through the
// shared-memory ring dominates), so the overhead term is a full strip's width.
constexpr int kMaxGrid = 2048;  // blocks of a launch
constexpr int kLaunches = 4;  // pass 1 (small tables), pass 1 (large tables), pass 2, detector only
// Pass 1's launches and pass 2 steal work (measured: with one precomputed run per block the SMs of
// the small tables' pass 1 sat 20 % idle -- a model cannot price every image of a mix); each needs
// its blocks' initial runs and the live copy the blocks claim from, kMaxGrid packed words each.
constexpr int kStealLaunches = 3;
constexpr int64_t kRowOverhead = 2048;

void partition(const JobDesc* J, int n, int SW, int grid, int64_t* starts)
{
    if (n == 0) {
        for (int k = 0; k <= grid; ++k) starts[k] = 0;
        return;
    }
    const JobDesc& last = J[n - 1];
    const int64_t u_end = last.unit_begin + (int64_t)last.bands * last.strips * last.H;
    double total = 0.0;
    for (int j = 0; j < n; ++j)
        for (int s = 0; s < J[j].strips; ++s)
            total += (double)J[j].bands * J[j].H * (double)(std::min(SW, J[j].W - s * SW) + kRowOverhead);
    const double per = total / grid;
    int k = 1;
    starts[0] = J[0].unit_begin;
    double acc = 0.0;
    for (int j = 0; j < n; ++j)
        for (int band = 0; band < J[j].bands; ++band)
            for (int s = 0; s < J[j].strips; ++s) {
                const double c = (double)(std::min(SW, J[j].W - s * SW) + kRowOverhead);
                const double seg = c * J[j].H;
                const int64_t u_seg = J[j].unit_begin + ((int64_t)band * J[j].strips + s) * J[j].H;
                while (k < grid && acc + seg >= per * k) {
                    int64_t rows = (int64_t)std::ceil((per * k - acc) / c);
                    rows = rows < 0 ? 0 : (rows > J[j].H ? J[j].H : rows);
                    starts[k] = std::max(starts[k - 1], u_seg + rows);
                    ++k;
                }
                acc += seg;
            }
    while (k <= grid) starts[k++] = u_end;
}

struct Plan {
    std::vector<int> kind;          // per job
    std::vector<size_t> fb_off;     // per job: workspace offset of a fallback job's own workspace
    std::vector<size_t> fb_bytes;
    std::vector<int64_t> tbl_first; // per job: first TableDesc index (TMA stretch jobs)
    int ns = 0, nd = 0, nbands_s = 0, nbands_d = 0;
    int ns_small = 0;  // stretch jobs of <= kSmallBits bits, placed first in the job table
    size_t off_sjobs = 0, off_djobs = 0, off_coef = 0, off_maps = 0, off_tables = 0, off_part = 0;
    size_t off_steal = 0;  // [kStealLaunches][2][kMaxGrid] uint64: initial runs, then the live runs
    size_t off_hist = 0, off_S = 0, off_lohi = 0, off_fb = 0, total = 0;
    size_t hist_bytes = 0, S_bytes = 0;
    int s_max_bits = 8, d_max_bits = 8;
};

// The start of every run: the stretch images' histograms cleared and each stealing launch's runs put
// back at their planned starts (the previous run left them used up) -- one kernel, where a memset and
// three copies would each leave a gap between the kernels around them.
struct ResetArgs {
    unsigned long long* hist;
    size_t hist_words;
    const uint64_t* init[kStealLaunches];
    unsigned long long* live[kStealLaunches];
    int count[kStealLaunches];
};

__global__ void __launch_bounds__(256) k_batch_reset(const ResetArgs a)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nt = (size_t)gridDim.x * blockDim.x;
    ulonglong2* h2 = reinterpret_cast<ulonglong2*>(a.hist);  // 256-byte aligned in the workspace
    const size_t pairs = a.hist_words / 2;
    for (size_t i = t; i < pairs; i += nt) h2[i] = make_ulonglong2(0ull, 0ull);
    if (t == 0 && (a.hist_words & 1)) a.hist[a.hist_words - 1] = 0ull;
#pragma unroll
    for (int l = 0; l < kStealLaunches; ++l)
        for (size_t i = t; i < (size_t)a.count[l]; i += nt) a.live[l][i] = a.init[l][i];
}

bool batch_tma_ok(const lutc_job& j)
{
    const lutc_raster& r = j.in;
    return r.width >= 256 && (int64_t)r.width * r.height > 0 && r.bits <= 15 && ((uintptr_t)r.data % 16 == 0) &&
           (r.pitch_bytes % 16 == 0) && (int64_t)r.bands * r.height < ((int64_t)1 << 31);
}

int check_job(const lutc_job& j)
{
    int rc = check_raster(&j.in);
    if (rc) return rc;
    if ((rc = check_coeff_set(&j.in, j.per_band))) return rc;
    if (j.flags & ~LUTC_STRETCH) return LUTC_EINVAL;
    const int64_t elem = (j.flags & LUTC_STRETCH) ? 1 : 2;
    if ((int64_t)j.in.width * j.in.height > 0 &&
        (!j.out || j.out_pitch_bytes < elem * j.in.width || j.out_pitch_bytes % elem))
        return LUTC_EINVAL;
    return LUTC_OK;
}

int make_plan(const lutc_job* jobs, int n, Plan& p)
{
    if (n < 0 || (n > 0 && !jobs)) return LUTC_EINVAL;
    p.kind.assign(n, kFallback);
    p.fb_off.assign(n, 0);
    p.fb_bytes.assign(n, 0);
    p.tbl_first.assign(n, -1);
    int64_t hist_elems = 0, S_bytes = 0;
    for (int i = 0; i < n; ++i) {
        int rc = check_job(jobs[i]);
        if (rc) return rc;
        const bool stretch = (jobs[i].flags & LUTC_STRETCH) != 0;
        if (batch_tma_ok(jobs[i])) {
            p.kind[i] = stretch ? kTmaStretch : kTmaDetector;
            if (stretch) {
                p.ns++;
                if (jobs[i].in.bits <= kSmallBits) p.ns_small++;
                p.nbands_s += jobs[i].in.bands;
                hist_elems += (int64_t)jobs[i].in.bands << jobs[i].in.bits;
                S_bytes += (int64_t)jobs[i].in.bands << jobs[i].in.bits;
                if (jobs[i].in.bits > p.s_max_bits) p.s_max_bits = jobs[i].in.bits;
            } else {
                p.nd++;
                p.nbands_d += jobs[i].in.bands;
                if (jobs[i].in.bits > p.d_max_bits) p.d_max_bits = jobs[i].in.bits;
            }
        } else if (stretch) {
            p.fb_bytes[i] = lutc_correct_image_workspace(&jobs[i].in);
        }
    }
    size_t o = 0;
    p.off_sjobs = o;
    o = align_up(o + sizeof(JobDesc) * p.ns, 256);
    p.off_djobs = o;
    o = align_up(o + sizeof(JobDesc) * p.nd, 256);
    p.off_coef = o;
    o = align_up(o + sizeof(BandCoef) * (p.nbands_s + p.nbands_d), 256);
    p.off_maps = o;
    o = align_up(o + sizeof(CUtensorMap) * (p.ns + p.nd), 256);
    p.off_tables = o;
    o = align_up(o + sizeof(TableDesc) * p.nbands_s, 256);
    p.off_part = o;
    o = align_up(o + sizeof(int64_t) * kLaunches * (kMaxGrid + 1), 256);
    p.off_steal = o;
    o = align_up(o + sizeof(uint64_t) * kStealLaunches * 2 * kMaxGrid, 256);
    p.off_hist = o;
    p.hist_bytes = (size_t)hist_elems * 8;
    o = align_up(o + p.hist_bytes, 256);
    p.off_S = o;
    p.S_bytes = (size_t)S_bytes;
    o = align_up(o + p.S_bytes, 256);
    p.off_lohi = o;
    o = align_up(o + (size_t)p.nbands_s * 8, 256);
    p.off_fb = o;
    for (int i = 0; i < n; ++i) {
        if (p.fb_bytes[i]) {
            p.fb_off[i] = o;
            o = align_up(o + p.fb_bytes[i], 256);
        }
    }
    p.total = o;
    return LUTC_OK;
}

}  // namespace

struct lutc_batch_st {
    std::vector<lutc_job> jobs;
    std::vector<std::vector<lutc_coeffs>> coefs;
    Plan plan;
    lutc_batch_config cfg;
    uint8_t* ws = nullptr;
    std::vector<uint8_t> blob;  // host image of the descriptor part of the workspace
    int64_t s_units = 0, d_units = 0;
    int64_t s_units_small = 0;  // units of the first ns_small stretch jobs
    int small_max_bits = 8;
    int grid[kLaunches] = {0, 0, 0, 0};
    bool steal = false;  // pass 1 and pass 2 steal work (unit numbers fit the packed runs)
    int granule[kLaunches] = {0, 0, 0, 0};  // units per claim of each stealing launch
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int default_tc(const std::vector<lutc_job>& jobs)
{
    // the narrowest image sets the strip width: a strip wider than an image idles threads
    int wmin = 1 << 30;
    for (const lutc_job& j : jobs)
        if (batch_tma_ok(j) && j.in.width < wmin) wmin = j.in.width;
    return wmin >= 4096 ? 256 : (wmin >= 1024 ? 128 : 64);
}

int enqueue(lutc_batch b, cudaStream_t st, cudaEvent_t* tr)
{
    const Plan& p = b->plan;
    int rc;
    if (tr) cudaEventRecord(tr[0], st);
    const int tc = b->cfg.column_threads;
    const int bps = b->cfg.blocks_per_sm;
    if (p.ns > 0) {
        BatchLaunch L;
        L.jobs = reinterpret_cast<const JobDesc*>(b->ws + p.off_sjobs);
        L.maps = reinterpret_cast<const CUtensorMap*>(b->ws + p.off_maps);
        L.njobs = p.ns;
        L.max_bits = p.s_max_bits;
        L.units = b->s_units;
        L.hist = reinterpret_cast<unsigned long long*>(b->ws + p.off_hist);
        L.S = b->ws + p.off_S;
        L.S_out = b->ws + p.off_S;
        L.unit_offset = 0;
        // pass 1 in two launches: small histograms (more blocks per SM), then the rest
        const int64_t* part = reinterpret_cast<const int64_t*>(b->ws + p.off_part);
        uint64_t* steal = reinterpret_cast<uint64_t*>(b->ws + p.off_steal);  // [launch][initial | live][block]
        {
            ResetArgs ra;
            ra.hist = L.hist;
            ra.hist_words = p.hist_bytes / 8;
            const bool runs[kStealLaunches] = {p.ns_small > 0, p.ns - p.ns_small > 0, true};
            for (int l = 0; l < kStealLaunches; ++l) {
                uint64_t* init = steal + (size_t)l * 2 * kMaxGrid;
                ra.init[l] = init;
                ra.live[l] = reinterpret_cast<unsigned long long*>(init + kMaxGrid);
                ra.count[l] = (b->steal && runs[l]) ? b->grid[l] : 0;
            }
            const size_t pairs = ra.hist_words / 2;
            const int blocks = (int)std::max<size_t>(1, std::min<size_t>((pairs + 255) / 256, (size_t)4 * sm_count()));
            k_batch_reset<<<blocks, 256, 0, st>>>(ra);
            if ((rc = cuda_status(cudaGetLastError()))) return rc;
        }
        BatchLaunch L1 = L;
        L1.njobs = p.ns_small;
        L1.max_bits = b->small_max_bits;
        L1.units = b->s_units_small;
        L1.starts = part;
        L1.grid = b->grid[0];
        BatchLaunch L2 = L;
        L2.jobs = L.jobs + p.ns_small;
        L2.maps = L.maps + p.ns_small;
        L2.njobs = p.ns - p.ns_small;
        L2.unit_offset = b->s_units_small;
        L2.units = b->s_units - b->s_units_small;
        L2.starts = part + (kMaxGrid + 1);
        L2.grid = b->grid[1];
        BatchLaunch* P1[2] = {&L1, &L2};
        for (int l = 0; l < 2; ++l) {
            BatchLaunch& Lp = *P1[l];
            if (Lp.njobs <= 0) continue;
            if (b->steal) {  // runs reset by k_batch_reset above
                Lp.ranges = reinterpret_cast<unsigned long long*>(steal + (size_t)l * 2 * kMaxGrid + kMaxGrid);
                Lp.granule = b->granule[l];
            }
            if ((rc = tma_batch_pass(Lp, kModeHist, tc, bps, st))) return rc;
        }
        if (tr) cudaEventRecord(tr[1], st);
        if ((rc = stretch_batch(reinterpret_cast<const TableDesc*>(b->ws + p.off_tables), p.nbands_s, L.hist,
                                b->ws + p.off_S, reinterpret_cast<int32_t*>(b->ws + p.off_lohi), st)))
            return rc;
        if (tr) cudaEventRecord(tr[2], st);
        L.starts = part + 2 * (kMaxGrid + 1);
        L.grid = b->grid[2];
        if (b->steal) {
            L.ranges = reinterpret_cast<unsigned long long*>(steal + (size_t)2 * 2 * kMaxGrid + kMaxGrid);
            L.granule = b->granule[2];
        }
        if ((rc = tma_batch_pass(L, kModeApplyStretch, tc, bps, st))) return rc;
    } else if (tr) {
        cudaEventRecord(tr[1], st);
        cudaEventRecord(tr[2], st);
    }
    if (p.nd > 0) {
        BatchLaunch L;
        L.jobs = reinterpret_cast<const JobDesc*>(b->ws + p.off_djobs);
        L.maps = reinterpret_cast<const CUtensorMap*>(b->ws + p.off_maps) + p.ns;
        L.njobs = p.nd;
        L.max_bits = p.d_max_bits;
        L.unit_offset = 0;
        L.units = b->d_units;
        L.starts = reinterpret_cast<const int64_t*>(b->ws + p.off_part) + 3 * (kMaxGrid + 1);
        L.grid = b->grid[3];
        L.hist = nullptr;
        L.S = nullptr;
        L.S_out = nullptr;
        if ((rc = tma_batch_pass(L, kModeApplyDetector, tc, bps, st))) return rc;
    }
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        if (p.kind[i] != kFallback) continue;
        const lutc_job& j = b->jobs[i];
        rc = lutc_correct_image(&j.in, b->coefs[i].data(), j.flags, j.out, j.out_pitch_bytes,
                                p.fb_bytes[i] ? b->ws + p.fb_off[i] : nullptr, p.fb_bytes[i], (lutc_stream)st);
        if (rc) return rc;
    }
    if (tr) cudaEventRecord(tr[3], st);
    return LUTC_OK;
}

void release_graph(lutc_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    b->exec = nullptr;
    b->graph = nullptr;
    b->cap = nullptr;
}

}  // namespace

extern "C" size_t lutc_batch_workspace(const lutc_job* jobs, int n)
{
    Plan p;
    if (make_plan(jobs, n, p)) return 0;
    return p.total;
}

extern "C" int lutc_batch_create(const lutc_job* jobs, int n, const lutc_batch_config* config, void* workspace,
                                 size_t workspace_bytes, lutc_stream stream, lutc_batch* out)
{
    if (!out) return LUTC_EINVAL;
    Plan p;
    int rc = make_plan(jobs, n, p);
    if (rc) return rc;
    if (p.total > 0 && (!workspace || workspace_bytes < p.total)) return LUTC_ENOMEM;
    if ((uintptr_t)workspace % 256) return LUTC_EINVAL;
    if (config && ((config->column_threads != 0 && config->column_threads != 64 && config->column_threads != 128 &&
                    config->column_threads != 256) ||
                   config->blocks_per_sm < 0 || config->blocks_per_sm > 32))
        return LUTC_EINVAL;

    lutc_batch b = new (std::nothrow) lutc_batch_st();
    if (!b) return LUTC_ENOMEM;
    b->jobs.assign(jobs, jobs + n);
    b->coefs.resize(n);
    for (int i = 0; i < n; ++i) {
        b->coefs[i].assign(jobs[i].per_band, jobs[i].per_band + jobs[i].in.bands);
        b->jobs[i].per_band = nullptr;
    }
    b->plan = p;
    b->cfg = config ? *config : lutc_batch_config{0, 0, 0};
    if (b->cfg.column_threads == 0) b->cfg.column_threads = default_tc(b->jobs);
    b->ws = reinterpret_cast<uint8_t*>(workspace);

    // descriptor image: job tables, coefficient pointers, tensor maps, table descriptors
    const int tc = b->cfg.column_threads;
    const int SW = 8 * tc;
    b->blob.assign(p.off_hist, 0);
    JobDesc* sj = reinterpret_cast<JobDesc*>(b->blob.data() + p.off_sjobs);
    JobDesc* dj = reinterpret_cast<JobDesc*>(b->blob.data() + p.off_djobs);
    BandCoef* cf = reinterpret_cast<BandCoef*>(b->blob.data() + p.off_coef);
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(b->blob.data() + p.off_maps);
    TableDesc* tbl = reinterpret_cast<TableDesc*>(b->blob.data() + p.off_tables);
    const BandCoef* d_cf = reinterpret_cast<const BandCoef*>(b->ws + p.off_coef);
    int is = 0, id = 0, icf = 0, it = 0;
    int64_t hist_off = 0, S_off = 0;
    // job table order: stretch jobs of <= kSmallBits bits, the other stretch jobs, then detector jobs
    std::vector<int> order;
    for (int pass = 0; pass < 3; ++pass)
        for (int i = 0; i < n; ++i) {
            if (p.kind[i] == kFallback) continue;
            const bool stretch = p.kind[i] == kTmaStretch;
            const bool small = b->jobs[i].in.bits <= kSmallBits;
            if ((pass == 0 && stretch && small) || (pass == 1 && stretch && !small) || (pass == 2 && !stretch))
                order.push_back(i);
        }
    for (int i : order) {
        const lutc_job& j = b->jobs[i];
        const bool stretch = p.kind[i] == kTmaStretch;
        JobDesc& J = stretch ? sj[is] : dj[id];
        J.W = j.in.width;
        J.H = j.in.height;
        J.bits = j.in.bits;
        J.bands = j.in.bands;
        J.strips = (j.in.width + SW - 1) / SW;
        const int64_t vec = stretch ? 8 : 16;
        J.vout = ((uintptr_t)j.out % vec == 0) && (j.out_pitch_bytes % vec == 0);
        int64_t& units = stretch ? b->s_units : b->d_units;
        J.unit_begin = units;
        units += (int64_t)J.bands * J.strips * J.H;
        J.out = reinterpret_cast<uint8_t*>(j.out);
        J.out_pitch = j.out_pitch_bytes;
        J.hist_off = stretch ? hist_off : 0;
        J.S_off = stretch ? S_off : 0;
        J.coef = d_cf + icf;
        for (int k = 0; k < j.in.bands; ++k)
            cf[icf++] = BandCoef{b->coefs[i][k].A, b->coefs[i][k].G, b->coefs[i][k].O};
        CUtensorMap* m = stretch ? &maps[is] : &maps[p.ns + id];
        if (!tma_encode(m, &j.in, tc)) {
            delete b;
            return LUTC_ECUDA;
        }
        if (stretch) {
            const int64_t L = (int64_t)1 << j.in.bits;
            b->plan.tbl_first[i] = it;
            if (is < p.ns_small) {
                b->s_units_small = b->s_units;
                if (j.in.bits > b->small_max_bits) b->small_max_bits = j.in.bits;
            }
            for (int k = 0; k < j.in.bands; ++k) {
                tbl[it].hist_off = hist_off + k * L;
                tbl[it].S_off = S_off + k * L;
                tbl[it].lohi_off = 2 * (int64_t)it;
                tbl[it].bits = j.in.bits;
                tbl[it].pad = 0;
                ++it;
            }
            hist_off += j.in.bands * L;
            S_off += j.in.bands * L;
            ++is;
        } else {
            ++id;
        }
    }
    // grids and cost-balanced block boundaries of the four launches
    {
        const int bps = b->cfg.blocks_per_sm;
        struct { const JobDesc* J; int n; int mode; int bits; } L[kLaunches] = {
            {sj, p.ns_small, kModeHist, b->small_max_bits},
            {sj + p.ns_small, p.ns - p.ns_small, kModeHist, p.s_max_bits},
            {sj, p.ns, kModeApplyStretch, p.s_max_bits},
            {dj, p.nd, kModeApplyDetector, p.d_max_bits}};
        int64_t* part = reinterpret_cast<int64_t*>(b->blob.data() + p.off_part);
        for (int l = 0; l < kLaunches; ++l) {
            int g = 0;
            if (L[l].n > 0) {
                g = tma_batch_grid(L[l].mode, tc, L[l].bits, bps);
                if (g <= 0) {
                    delete b;
                    return LUTC_ECUDA;
                }
                g = std::min(g, kMaxGrid);
            }
            b->grid[l] = g;
            partition(L[l].J, L[l].n, SW, std::max(g, 1), part + (size_t)l * (kMaxGrid + 1));
        }
        // the stealing launches' initial runs as packed (start << 32 | end) words, when every unit number
        // fits, and their claim size: about a sixteenth of a block's share in whole tiles, one to eight
        // (a claim costs one atomic round trip; the last claims set how evenly the blocks finish)
        b->steal = b->s_units < kStealMaxUnits;
        uint64_t* steal = reinterpret_cast<uint64_t*>(b->blob.data() + p.off_steal);
        const int64_t units_of[kStealLaunches] = {b->s_units_small, b->s_units - b->s_units_small, b->s_units};
        const int64_t rt = tma_box_rows(tc);
        for (int l = 0; l < kStealLaunches && b->steal; ++l) {
            const int64_t* st0 = part + (size_t)l * (kMaxGrid + 1);
            for (int k = 0; k < b->grid[l]; ++k)
                steal[(size_t)l * 2 * kMaxGrid + k] = ((uint64_t)st0[k] << 32) | (uint64_t)st0[k + 1];
            const int64_t per_block = b->grid[l] > 0 ? units_of[l] / b->grid[l] : 0;
            b->granule[l] = (int)(rt * std::min<int64_t>(8, std::max<int64_t>(1, per_block / (16 * rt))));
        }
    }
    if (p.off_hist > 0) {
        rc = cuda_status(cudaMemcpyAsync(b->ws, b->blob.data(), p.off_hist, cudaMemcpyHostToDevice,
                                         (cudaStream_t)stream));
        if (rc) {
            delete b;
            return rc;
        }
    }
    *out = b;
    return LUTC_OK;
}

extern "C" int lutc_batch_run(lutc_batch b, lutc_stream stream)
{
    if (!b) return LUTC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->cfg.use_graph) return enqueue(b, st, trace_slot());
    if (!b->exec) {
        int rc;
        if ((rc = cuda_status(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)))) return rc;
        if ((rc = cuda_status(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)))) {
            release_graph(b);
            return rc;
        }
        const int erc = enqueue(b, b->cap, nullptr);
        const cudaError_t end = cudaStreamEndCapture(b->cap, &b->graph);
        if (erc || end != cudaSuccess) {
            cudaGetLastError();
            release_graph(b);
            return erc ? erc : LUTC_ECUDA;
        }
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
            cudaGetLastError();
            release_graph(b);
            return LUTC_ECUDA;
        }
    }
    return cuda_status(cudaGraphLaunch(b->exec, st));
}

extern "C" int lutc_batch_correct(const lutc_job* jobs, int n, const lutc_batch_config* config, void* workspace,
                                  size_t workspace_bytes, lutc_stream stream)
{
    lutc_batch_config c = config ? *config : lutc_batch_config{0, 0, 0};
    c.use_graph = 0;  // one run: a graph would only add its capture
    lutc_batch b = nullptr;
    int rc = lutc_batch_create(jobs, n, &c, workspace, workspace_bytes, stream, &b);
    if (rc) return rc;
    rc = lutc_batch_run(b, stream);
    lutc_batch_destroy(b);  // host state only: the enqueued work keeps nothing of it
    return rc;
}

extern "C" int lutc_batch_tables(lutc_batch b, int job, uint64_t** hist, uint8_t** S, int32_t** lohi)
{
    if (!b || job < 0 || job >= (int)b->jobs.size()) return LUTC_EINVAL;
    const Plan& p = b->plan;
    const lutc_job& j = b->jobs[job];
    if (!(j.flags & LUTC_STRETCH)) return LUTC_EINVAL;
    if (p.kind[job] == kTmaStretch) {
        // locate the job's tables from its first table descriptor
        const TableDesc* tbl = reinterpret_cast<const TableDesc*>(b->blob.data() + p.off_tables);
        const TableDesc& t = tbl[p.tbl_first[job]];
        if (hist) *hist = reinterpret_cast<uint64_t*>(b->ws + p.off_hist) + t.hist_off;
        if (S) *S = b->ws + p.off_S + t.S_off;
        if (lohi) *lohi = reinterpret_cast<int32_t*>(b->ws + p.off_lohi) + t.lohi_off;
        return LUTC_OK;
    }
    size_t ho = 0, so = 0, lo = 0;
    int rc = lutc_correct_image_tables(&j.in, &ho, &so, &lo);
    if (rc) return rc;
    uint8_t* w = b->ws + p.fb_off[job];
    if (hist) *hist = reinterpret_cast<uint64_t*>(w + ho);
    if (S) *S = w + so;
    if (lohi) *lohi = reinterpret_cast<int32_t*>(w + lo);
    return LUTC_OK;
}

extern "C" int lutc_batch_destroy(lutc_batch b)
{
    if (!b) return LUTC_EINVAL;
    release_graph(b);
    delete b;
    return LUTC_OK;
}

extern "C" int lutc_batch_autotune(const lutc_job* jobs, int n, void* workspace, size_t workspace_bytes,
                                   lutc_stream stream, int reps, lutc_batch_config* best, float* best_ms)
{
    if (!best || reps < 1) return LUTC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LUTC_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LUTC_ECUDA;
    }
    static const int kTc[3] = {64, 128, 256};
    static const int kBps[2] = {0, 2};
    float best_t = -1.0f;
    int rc = LUTC_OK;
    for (int a = 0; a < 3 && rc == LUTC_OK; ++a) {
        for (int c = 0; c < 2 && rc == LUTC_OK; ++c) {
            const lutc_batch_config cfg = {kTc[a], kBps[c], 0};
            lutc_batch b = nullptr;
            if ((rc = lutc_batch_create(jobs, n, &cfg, workspace, workspace_bytes, stream, &b))) break;
            rc = lutc_batch_run(b, stream);  // warm-up
            if (!rc) rc = cuda_status(cudaEventRecord(e0, st));
            for (int r = 0; r < reps && !rc; ++r) rc = lutc_batch_run(b, stream);
            if (!rc) rc = cuda_status(cudaEventRecord(e1, st));
            if (!rc) rc = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.0f;
            if (!rc) rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
            lutc_batch_destroy(b);
            ms /= (float)reps;
            if (!rc && (best_t < 0.0f || ms < best_t)) {
                best_t = ms;
                *best = cfg;
                best->use_graph = 1;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc && best_ms) *best_ms = best_t;
    return rc;
}
