// api.cu -- the C-ABI of include/metade.h: context creation and validation,
// the descriptor table, the launch planner (kernel kind per executor, work
// order, block shape), CUDA-graph capture of whole evolver generations, and
// the sticky device status.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/metade.h"
#include "internal.h"

using namespace metade;

namespace {

constexpr int kMaxDim = 1536;
// Reduced-precision executors at least this wide use the tensor cores unless
// the configuration fixes another width: 129 is the first D whose padded row
// (D_pad > 128) no longer lets the fused tile kernel keep R^T in shared memory.
constexpr int kTcDefaultMinDim = 129;
constexpr int kTcAltMinDim = 256;  // the widths metade_autotune also tries: every executor wider than the
constexpr int kTcLowMinDim = 33;   // small-D kernel's reach, and only those of 256 and more
// FP32: executors with D >= the width (or D_pad > 256) run the per-generation pipeline with the FP32
// GEMM on the CUDA cores (k_rot_simt); the fused kernels keep the others.  257 unless set or tuned.
constexpr int kSimtDefaultMinDim = 257;
constexpr int kMaxNp = 1024;
constexpr size_t kSmemLimit = 227 * 1024;

struct Bucket {
    FusedPlan plan;
    int work_off, n_work;
    std::string tuned;  // autotuner record: candidate threads -> ms
};

enum ProfKind {
    kProfFusedSmall = 0,
    kProfFusedGeneral = 1,
    kProfTcGemm = 2,
    kProfTcGeneration = 3,
    kProfFusedTileStream = 4,
    kProfFusedTile = 5,
    kProfFusedMlp = 6,
    kProfTcPrologue = 7,
    kProfTcTrial = 8,
    kProfTcSelect = 9,
    kProfTcTies = 10,
    kProfTcSel = 11,
    kProfNearTies = 12,  // a count only: selections decided by the near-tie path
    kProfKinds = 13
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

struct GraphEntry {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    int64_t kernels;
};

}  // namespace

struct metade_ctx {
    // configuration (host copies)
    int n_prob = 0, n_inst = 0, n_groups = 0, n_out = 0;
    float lo = -100.f, hi = 100.f;
    uint64_t seed = 0;
    int one_shot = 0, p_best_pct = 10;
    metade_prec prec = METADE_FP32;
    metade_path path = METADE_PATH_BATCHED;
    int tie_fp64 = 0;
    int evolver = 0;  // 0 DE/rand/1/bin (Alg. 3), 1 PSO, 2 CSO, 3 NES (xNES)
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;  // private stream for graph capture
    static constexpr int kSide = 3;
    cudaStream_t side[kSide] = {};  // forked streams: size buckets run beside the per-generation pipelines
    cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
    std::vector<InstDesc> hdesc;
    std::vector<long long> pop_off;
    std::vector<long long> fit_off;
    std::vector<int> dpad;
    long long pop_floats = 0, n_indiv = 0;
    int max_np = 0, max_dim = 0, max_dpad = 0, max_kp = 1;
    // device
    InstDesc* desc = nullptr;
    int* row_inst = nullptr;
    float* rot = nullptr;
    float* rotT = nullptr;
    float* shift = nullptr;
    float* uscr = nullptr;
    float* fuscr = nullptr;
    int* topk = nullptr;
    int* status = nullptr;
    uint32_t* gen_dev = nullptr;
    unsigned* bar = nullptr;  // plain path: grid-barrier arrival count
    int* work = nullptr;
    std::vector<Bucket> buckets;
    std::vector<GraphEntry> graphs;
    int64_t launches = 0;
    bool prof_on = false;
    int prof_stride = 1;       // profiling: one tensor-core generation in prof_stride records its events
    long long prof_gen = 0;    // tensor-core generations enqueued while profiling, for the sampling
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> prof_events;  // every event the records refer to (destroyed on read)
    // large-D executors on the tensor cores (prec BF16 / BF16X3)
    int tc_min_dim = kTcDefaultMinDim;  // executors with D >= this run on the GEMM pipeline
    int tc_unfused = 0;                 // 1: the per-kernel pipeline even where the fused kernel applies
    bool tc_auto = false;               // metade_autotune picks tc_min_dim
    std::string tc_tuned;               // autotuner record: width -> ms
    bool tc = false;
    TcPlan tcp;
    std::vector<char> is_tc;
    int* tc_execs = nullptr;
    int* tc_row_exec = nullptr;
    int* tc_tiles = nullptr;
    long long* tc_brow = nullptr;
    int* tc_topk = nullptr;
    int* tc_ties = nullptr;
    int* tc_tp = nullptr;  // problem -> path index, first rows, tie counts
    long long* tc_tie_off = nullptr;  // population offsets of listed near ties
    int4* tc_trec = nullptr;          // per operand row: draw record (k_tc_rank -> k_tc_trial2, k_tc_sel)
    int4* tc_tmeta = nullptr;         // per tensor-core tile: first row, rows, D, D_pad, objective, problem
    unsigned long long* tie_total = nullptr;  // near ties decided by the tensor-core path since the last read
    int* tc_tie_done = nullptr;       // wide four-kernel generation: row groups finished per tie chunk
    float* tc_tie_zs = nullptr;       // wide four-kernel generation: z and dz of each listed tie
    uint8_t *aq = nullptr, *aq_lo = nullptr, *bq = nullptr, *bq_lo = nullptr;  // BF16 pairs or e4m3 bytes
    float *ascale = nullptr, *bscale = nullptr;                                // FP8 dequantisation factors
    unsigned* amax = nullptr;                                                  // FP8: max|R| scratch
    float *mlp_x = nullptr, *mlp_y = nullptr;  // MLP objective: inputs [256][16], targets per problem [256][2]
    MlpPlan mlpp{};                             // MLP executors' rows (n_rows 0: none)
    int *mlp_execs = nullptr, *mlp_row_exec = nullptr, *mlp_topk = nullptr;
};

namespace {

thread_local cudaError_t g_last_cuda = cudaSuccess;  // behind the last METADE_ECUDA of this thread

metade_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return METADE_OK;
    g_last_cuda = e;
    return METADE_ECUDA;
}

#define CK(x)                                                \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) return cuda_status(e_);       \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

StepArgs step_args(metade_ctx* c, float* pop, float* fit, const float* theta, uint32_t epoch,
                   const uint32_t* epoch_dev, uint32_t gen0, int n_gens, float* best_f, int* best_i) {
    StepArgs a;
    a.desc = c->desc;
    a.pop = pop;
    a.fit = fit;
    a.theta = theta;
    a.rot = c->rot;
    a.rotT = c->rotT;
    a.shift = c->shift;
    a.key = make_key(c->seed, kTagInner);
    a.epoch = epoch;
    a.epoch_dev = epoch_dev;
    a.gen0 = gen0;
    a.n_gens = n_gens;
    a.lo = c->lo;
    a.hi = c->hi;
    a.best_f = best_f;
    a.best_i = best_i;
    a.status = c->status;
    a.tie_fp64 = c->tie_fp64;
    return a;
}

double work_cost(const InstDesc& d) { return (double)d.np * ((double)d.dim * d.dim + 16.0 * d.dim + 64.0); }

static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Order of a small-D bucket: when the bucket has more executors than the GPU
// has SMs, the executors that share an SM (one wave: blocks w, w + n_SM,
// w + 2 n_SM, ... land on one SM, as measured on GB300 with %smid) are made
// to share an objective, so the resident CTAs of an SM run the same branch of
// the objective code and compete less for instruction cache.  Any order is
// correct (each executor's result depends only on its own state and draws);
// this one is faster (8.85 -> 8.67 ms per 500 generations of the 600-executor
// D = 20 workload).
static void cohere_by_objective(const metade_ctx* c, std::vector<int>& v) {
    const int n = (int)v.size(), nsm = device_sms();
    if (nsm <= 0 || n <= nsm) return;
    std::vector<int> L = v;
    std::stable_sort(L.begin(), L.end(), [&](int x, int y) { return c->hdesc[x].obj < c->hdesc[y].obj; });
    int j = 0;
    for (int sm = 0; sm < nsm; ++sm)
        for (int w = sm; w < n; w += nsm) v[w] = L[j++];
}

// Kernel kind per executor and the work order inside each bucket (largest
// first, so the block scheduler hands the longest executors out first; small-D
// buckets then grouped by objective per SM).
metade_status build_plan(metade_ctx* c) {
    std::vector<std::vector<int>> small(33);
    std::vector<int> general, tile, tile_stream;
    for (int k = 0; k < c->n_inst; ++k) {
        if (c->tc && c->is_tc[k]) continue;
        const InstDesc& d = c->hdesc[k];
        if (d.obj == kMlp) continue;  // the MLP objective has its own per-generation path
        const int dm = small_dmax_for(d.dim);
        // The tile kernels decide near ties by the FP32 difference form only;
        // FP64 tie re-evaluation runs in the small and general kernels.
        const bool fp32_ties = !c->tie_fp64;
        if (dm > 0 && fused_smem_small(dm, d.np) <= kSmemLimit) small[dm].push_back(k);
        else if (fp32_ties && d.dpad <= 128 && fused_smem_tile(d.np, d.dpad, 256, true) <= kSmemLimit) tile.push_back(k);
        else if (fp32_ties && d.dpad <= 256 && fused_smem_tile(d.np, d.dpad, 256, false) <= kSmemLimit)
            tile_stream.push_back(k);
        else general.push_back(k);
    }
    std::vector<int> order;
    auto sort_desc = [&](std::vector<int>& v) {
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return work_cost(c->hdesc[a]) > work_cost(c->hdesc[b]); });
    };
    c->buckets.clear();
    for (int dm = 1; dm <= 32; ++dm) {
        if (small[dm].empty()) continue;
        sort_desc(small[dm]);
        cohere_by_objective(c, small[dm]);
        int mnp = 0;
        for (int k : small[dm]) mnp = std::max(mnp, c->hdesc[k].np);
        Bucket b;
        b.plan.kind = 0;
        b.plan.dmax = dm;
        b.plan.threads = std::min(256, std::max(32, (mnp + 31) / 32 * 32));
        b.plan.grid = (int)small[dm].size();
        b.plan.smem = fused_smem_small(dm, mnp);
        b.plan.rot_smem = 0;
        b.plan.pop_smem = 1;
        b.plan.max_np = mnp;
        b.plan.max_dpad = dm;
        b.work_off = (int)order.size();
        b.n_work = (int)small[dm].size();
        order.insert(order.end(), small[dm].begin(), small[dm].end());
        c->buckets.push_back(b);
    }
    // tile buckets: R^T resident (D_pad <= 128) and streamed (D_pad <= 256)
    for (int mode = 1; mode >= 0; --mode) {
        std::vector<int>& tv = mode ? tile : tile_stream;
        if (tv.empty()) continue;
        sort_desc(tv);
        int mnp = 0, mdp = 0;
        for (int k : tv) {
            mnp = std::max(mnp, c->hdesc[k].np);
            mdp = std::max(mdp, c->hdesc[k].dpad);
        }
        Bucket b;
        b.plan.kind = 3;
        b.plan.dmax = 0;
        b.plan.threads = 256;
        b.plan.grid = (int)tv.size();
        b.plan.max_np = mnp;
        b.plan.max_dpad = mdp;
        b.plan.rot_smem = mode;
        b.plan.pop_smem = 0;
        b.plan.smem = fused_smem_tile(mnp, mdp, 256, mode != 0);
        if (b.plan.smem > kSmemLimit) return METADE_EUNSUPPORTED;
        b.work_off = (int)order.size();
        b.n_work = (int)tv.size();
        order.insert(order.end(), tv.begin(), tv.end());
        c->buckets.push_back(b);
    }
    if (!general.empty()) {
        sort_desc(general);
        int mnp = 0, mdp = 0;
        for (int k : general) {
            mnp = std::max(mnp, c->hdesc[k].np);
            mdp = std::max(mdp, c->hdesc[k].dpad);
        }
        Bucket b;
        b.plan.kind = 1;
        b.plan.dmax = 0;
        b.plan.threads = 256;
        b.plan.grid = (int)general.size();
        b.plan.max_np = mnp;
        b.plan.max_dpad = mdp;
        b.plan.rot_smem = fused_smem_general(mnp, mdp, 256, true) <= kSmemLimit ? 1 : 0;
        b.plan.pop_smem = 0;
        b.plan.smem = fused_smem_general(mnp, mdp, 256, b.plan.rot_smem != 0);
        if (b.plan.smem > kSmemLimit) return METADE_EUNSUPPORTED;
        b.work_off = (int)order.size();
        b.n_work = (int)general.size();
        order.insert(order.end(), general.begin(), general.end());
        c->buckets.push_back(b);
    }
    cudaFree(c->work);
    c->work = nullptr;
    if (!order.empty()) {
        CK(dalloc(&c->work, order.size()));
        CK(cudaMemcpy(c->work, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    return METADE_OK;
}

// Release the tensor-core pipeline's buffers (before re-planning, or at destroy).
void free_tc(metade_ctx* c) {
    cudaFree(c->tc_execs);
    cudaFree(c->tc_row_exec);
    cudaFree(c->tc_tiles);
    cudaFree(c->tc_brow);
    cudaFree(c->tc_topk);
    cudaFree(c->tc_ties);
    cudaFree(c->aq);
    cudaFree(c->aq_lo);
    cudaFree(c->bq);
    cudaFree(c->bq_lo);
    cudaFree(c->ascale);
    cudaFree(c->bscale);
    cudaFree(c->amax);
    cudaFree(c->tc_tp);
    cudaFree(c->tc_tie_off);
    cudaFree(c->tc_trec);
    cudaFree(c->tc_tmeta);
    c->tc_trec = nullptr;
    c->tc_tmeta = nullptr;
    cudaFree(c->tc_tie_done);
    cudaFree(c->tc_tie_zs);
    c->tc_tp = nullptr;
    c->tc_tie_off = nullptr;
    c->tc_tie_done = nullptr;
    c->tc_tie_zs = nullptr;
    c->tc_execs = c->tc_row_exec = c->tc_tiles = c->tc_topk = c->tc_ties = nullptr;
    c->tc_brow = nullptr;
    c->aq = c->aq_lo = c->bq = c->bq_lo = nullptr;
    c->ascale = c->bscale = nullptr;
    c->amax = nullptr;
    c->tc = false;
    c->tcp = TcPlan{};
    c->is_tc.assign(c->n_inst, 0);
}

// Executors on the per-generation GEMM pipeline: with BF16 / bf16x3 / FP8,
// every executor with D >= tc_min_dim (tensor cores); with FP32, the ones
// with D >= tc_min_dim and every one too wide for the tile kernels (D_pad >
// 256), with the GEMM on the CUDA cores.  Their operand
// rows are ordered by problem, then executor (InstDesc.tc_row = first row),
// so that a 128-row M tile of the tensor-core GEMM can span consecutive
// executors of one problem: they share the B operand (the problem's R), and
// the tiles stay full however small each population is.  The FP32 GEMM keeps
// 64-row tiles per executor.  Re-uploads the descriptor table.
metade_status setup_tc(metade_ctx* c) {
    free_tc(c);
    for (InstDesc& d : c->hdesc)
        if (d.obj != kMlp) {
            d.on_tc = 0;
            d.tc_row = 0;
        }
    const bool fp8 = c->prec == METADE_FP8E4M3;
    const bool simt = c->prec == METADE_FP32 && c->path == METADE_PATH_BATCHED;
    const bool reduced = c->prec == METADE_BF16 || c->prec == METADE_BF16X3 || fp8;
    const int kalign = fp8 ? 128 : 64;  // K elements per 128-byte operand tile (unused by the FP32 GEMM)
    std::vector<int> tc_execs, tc_row_exec, tc_tiles;
    std::vector<int> prob_tp(c->n_prob, -1), tp_row0;  // problems on the path, their first rows
    std::vector<long long> tc_brow(c->n_prob, -1);
    long long tc_brows = 0;
    int tc_kp = 0, tc_max_dpad = 0;
    if (reduced || simt) {
        for (int k = 0; k < c->n_inst; ++k) {
            const InstDesc& d = c->hdesc[k];
            if (d.obj == kMlp || (d.dim < c->tc_min_dim && (!simt || d.dpad <= 256))) continue;
            tc_execs.push_back(k);
        }
        // by problem, the widest problems first: the kernels that hand out rows, tiles or tie chunks
        // in this order start the costliest work first, and the generation's tail is the cheapest
        std::stable_sort(tc_execs.begin(), tc_execs.end(), [&](int x, int y) {
            const InstDesc &dx = c->hdesc[x], &dy = c->hdesc[y];
            return dx.dim != dy.dim ? dx.dim > dy.dim : dx.prob < dy.prob;
        });
        int prob_row0 = 0;  // first operand row of the current problem
        for (size_t q = 0; q < tc_execs.size(); ++q) {
            const int k = tc_execs[q];
            InstDesc& d = c->hdesc[k];
            c->is_tc[k] = 1;
            d.tc_row = (int)tc_row_exec.size();
            d.on_tc = 1;
            for (int i = 0; i < d.np; ++i) tc_row_exec.push_back(k);
            if (simt)
                for (int m0 = 0; m0 < d.np; m0 += 64) {
                    tc_tiles.push_back(k);
                    tc_tiles.push_back(m0);
                }
            tc_kp = std::max(tc_kp, (d.dim + kalign - 1) / kalign * kalign);
            tc_max_dpad = std::max(tc_max_dpad, d.dpad);
            if (tc_brow[d.prob] < 0) {
                tc_brow[d.prob] = tc_brows;
                tc_brows += (d.dim + 255) / 256 * 256;
            }
            // tensor cores: (first row, rows) tiles over the problem's rows, cut after its last executor
            if (q == 0 || c->hdesc[tc_execs[q - 1]].prob != d.prob) {
                prob_row0 = d.tc_row;
                prob_tp[d.prob] = (int)tp_row0.size();
                tp_row0.push_back(prob_row0);
            }
            const bool last_of_prob = q + 1 == tc_execs.size() || c->hdesc[tc_execs[q + 1]].prob != d.prob;
            if (!simt && last_of_prob) {
                const int r0 = prob_row0, r1 = (int)tc_row_exec.size();
                for (int r = r0; r < r1; r += 128) {
                    tc_tiles.push_back(r);
                    tc_tiles.push_back(std::min(128, r1 - r));
                }
            }
        }
        c->tc = !tc_execs.empty();
    }
    if (c->n_inst > 0 &&
        cudaMemcpy(c->desc, c->hdesc.data(), sizeof(InstDesc) * c->n_inst, cudaMemcpyHostToDevice) != cudaSuccess)
        return METADE_ECUDA;
    if (!c->tc) return METADE_OK;
    const bool split = c->prec == METADE_BF16X3;
    const size_t nrows = tc_row_exec.size();
    const size_t esz = fp8 ? 1 : 2;  // operand element bytes
    if (dalloc(&c->tc_execs, tc_execs.size()) || dalloc(&c->tc_row_exec, nrows) ||
        dalloc(&c->tc_tiles, tc_tiles.size()) || dalloc(&c->tc_brow, (size_t)c->n_prob) ||
        dalloc(&c->tc_topk, (size_t)c->n_indiv) || dalloc(&c->tc_ties, nrows + 2) ||
        (!simt && (dalloc(&c->aq, nrows * tc_kp * esz) || dalloc(&c->bq, (size_t)tc_brows * tc_kp * esz))) ||
        (split && (dalloc(&c->aq_lo, nrows * tc_kp * esz) || dalloc(&c->bq_lo, (size_t)tc_brows * tc_kp * esz))) ||
        (fp8 && (dalloc(&c->ascale, nrows) || dalloc(&c->bscale, (size_t)c->n_prob) || dalloc(&c->amax, 1))) ||
        dalloc(&c->tc_tp, (size_t)c->n_prob + 2 * tp_row0.size() + 1) || dalloc(&c->tc_tie_off, nrows) ||
        dalloc(&c->tc_trec, 4 * nrows) || (!simt && dalloc(&c->tc_tmeta, tc_tiles.size())))
        return METADE_ENOMEM;
    if (!simt) {  // the tile table k_tc_sel reads: two int4 per tile
        std::vector<int4> tm(tc_tiles.size());
        for (size_t q = 0; q < tc_tiles.size() / 2; ++q) {
            const InstDesc& d = c->hdesc[tc_row_exec[tc_tiles[2 * q]]];
            tm[2 * q] = make_int4(tc_tiles[2 * q], tc_tiles[2 * q + 1], d.dim, d.dpad);
            tm[2 * q + 1] = make_int4(d.obj, d.prob, 0, 0);
        }
        if (cudaMemcpy(c->tc_tmeta, tm.data(), sizeof(int4) * tm.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return METADE_ECUDA;
    }
    const int sel_ctas = std::max(1, device_sms());
    std::vector<int> tp_host(prob_tp);
    tp_host.insert(tp_host.end(), tp_row0.begin(), tp_row0.end());
    tp_host.resize((size_t)c->n_prob + 2 * tp_row0.size() + 1, 0);
    if (cudaMemcpy(c->tc_tp, tp_host.data(), sizeof(int) * tp_host.size(), cudaMemcpyHostToDevice))
        return METADE_ECUDA;
    if (cudaMemcpy(c->tc_execs, tc_execs.data(), sizeof(int) * tc_execs.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->tc_row_exec, tc_row_exec.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->tc_tiles, tc_tiles.data(), sizeof(int) * tc_tiles.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->tc_brow, tc_brow.data(), sizeof(long long) * c->n_prob, cudaMemcpyHostToDevice))
        return METADE_ECUDA;
    if (!simt) {
        std::vector<char> packed(c->n_prob, 0);
        for (int k : tc_execs) {
            const InstDesc& d = c->hdesc[k];
            if (packed[d.prob]) continue;
            packed[d.prob] = 1;
            if (launch_tc_pack_rot(c->rot, d.rot_off, d.dim, d.dpad, tc_kp, (d.dim + 255) / 256 * 256, c->bq,
                                   split ? c->bq_lo : nullptr, tc_brow[d.prob], fp8 ? 1 : 0, c->amax,
                                   fp8 ? c->bscale + d.prob : nullptr, c->st))
                return METADE_ECUDA;
            c->launches += 1;
        }
    }
    if (cudaStreamSynchronize(c->st)) return METADE_ECUDA;
    TcPlan& t = c->tcp;
    t.execs = c->tc_execs;
    t.n_exec = (int)tc_execs.size();
    t.row_exec = c->tc_row_exec;
    t.n_rows = (int)nrows;
    t.tiles = c->tc_tiles;
    t.n_tiles = (int)tc_tiles.size() / 2;
    t.brow = c->tc_brow;
    t.topk_all = c->tc_topk;
    t.uscr = c->uscr;
    t.fu = c->fuscr;
    t.aq = c->aq;
    t.aq_lo = c->aq_lo;
    t.bq = c->bq;
    t.bq_lo = c->bq_lo;
    t.ascale = c->ascale;
    t.bscale = c->bscale;
    t.fp8 = fp8 ? 1 : 0;
    t.simt = simt ? 1 : 0;
    t.tie_list = c->tc_ties + 2;
    t.tie_count = c->tc_ties;
    t.next_tile = c->tc_ties + 1;
    t.tie_off = c->tc_tie_off;
    t.trial_rec = c->tc_trec;
    t.tmeta = c->tc_tmeta;
    t.n_tp = (int)tp_row0.size();
    t.prob_tp = c->tc_tp;
    t.tp_row0 = c->tc_tp + c->n_prob;
    t.tie_cnt = c->tc_tp + c->n_prob + t.n_tp;
    t.chunk_ctr = c->tc_tp + c->n_prob + 2 * t.n_tp;
    t.tie_ctas = std::max(1, device_sms()) * 2;
    t.kp = tc_kp;
    t.split = split ? 1 : 0;
    t.max_dpad = tc_max_dpad;
    // BF16 with FP32 difference-form ties: four kernels per generation (ranking,
    // trial rows, GEMM with selection and commit, near ties); the persistent
    // k_tc_sel holds operands of at most 256 elements, k_rot_tc selects for wider ones
    if (c->prec == METADE_BF16 && !c->tie_fp64 && !c->tc_unfused) t.fused = tc_fused_fits(tc_kp) ? 1 : 2;
    else t.fused = 0;
    t.gen_ctas = sel_ctas;
    if (!c->tie_total) {  // kept across plans: the count runs until the next profile read
        if (dalloc(&c->tie_total, 1)) return METADE_ENOMEM;
        if (cudaMemset(c->tie_total, 0, sizeof(unsigned long long)) != cudaSuccess) return METADE_ECUDA;
    }
    t.tie_total = c->tie_total;
    t.tie_done = nullptr;
    t.tie_zs = nullptr;
    t.wide_ctas = 0;
    if (!c->tie_fp64 && tc_max_dpad > 256) {  // the row-split tie kernel's scratch: chunk counters, z and dz
        const size_t vs = (size_t)((tc_max_dpad + 3) & ~3);
        if (dalloc(&c->tc_tie_done, nrows) || dalloc(&c->tc_tie_zs, nrows * 2 * vs)) return METADE_ENOMEM;
        if (cudaMemset(c->tc_tie_done, 0, sizeof(int) * nrows) != cudaSuccess) return METADE_ECUDA;
        t.tie_done = c->tc_tie_done;
        t.tie_zs = c->tc_tie_zs;
        t.wide_ctas = tc_ties_wide_ctas(tc_max_dpad);
        if (t.wide_ctas <= 0) return METADE_ECUDA;
    }

    // a tie keeps four rows of max_dpad in shared memory (FP64 with tie_fp64)
    if ((size_t)4 * tc_max_dpad * (c->tie_fp64 ? sizeof(double) : sizeof(float)) > kSmemLimit)
        return METADE_EUNSUPPORTED;
    if (simt) {
        // no operands, no tensor maps: k_rot_simt reads the trial rows and R^T itself
    } else if (!tc_make_map(&t.mapA, c->aq, (long long)nrows, tc_kp, 128, (int)esz) ||
               !tc_make_map(&t.mapB, c->bq, tc_brows, tc_kp, 256, (int)esz) ||
               (split && (!tc_make_map(&t.mapAlo, c->aq_lo, (long long)nrows, tc_kp, 128, (int)esz) ||
                          !tc_make_map(&t.mapBlo, c->bq_lo, tc_brows, tc_kp, 256, (int)esz)))) {
        return METADE_ECUDA;
    }
    if (!split && !simt) {
        t.mapAlo = t.mapA;
        t.mapBlo = t.mapB;
    }
    return METADE_OK;
}

// Event pair around a launch when profiling is on (never inside a capture).
bool prof_pair(metade_ctx* c, cudaStream_t st, int kind, cudaEvent_t* a, cudaEvent_t* b) {
    *a = *b = nullptr;
    if (!c->prof_on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (cudaEventCreate(a) != cudaSuccess) return false;
    if (cudaEventCreate(b) != cudaSuccess) {
        cudaEventDestroy(*a);
        return false;
    }
    c->prof_events.push_back(*a);
    c->prof_events.push_back(*b);
    c->prof.push_back(ProfRec{kind, *a, *b});
    return true;
}

// Events between the kernels of one tensor-core generation (prologue, trial,
// GEMM, selection, ties): ev[0..5], with a record per kernel and one for the
// whole generation.
// The four-kernel generation has five events: ranking, trial, selection, ties.
bool prof_tc(metade_ctx* c, cudaStream_t st, cudaEvent_t* ev, bool fused) {
    if (!c->prof_on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    const int n = fused ? 5 : 6;
    for (int i = 0; i < n; ++i) {
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return false;
        }
    }
    for (int i = 0; i < n; ++i) c->prof_events.push_back(ev[i]);
    const int kinds[5] = {kProfTcPrologue, kProfTcTrial, kProfTcGemm, kProfTcSelect, kProfTcTies};
    const int fkinds[4] = {kProfTcPrologue, kProfTcTrial, kProfTcSel, kProfTcTies};
    for (int i = 0; i < n - 1; ++i) c->prof.push_back(ProfRec{fused ? fkinds[i] : kinds[i], ev[i], ev[i + 1]});
    c->prof.push_back(ProfRec{kProfTcGeneration, ev[0], ev[n - 1]});
    return true;
}

metade_status run_inner(metade_ctx* c, cudaStream_t st, float* pop, float* fit, const float* theta, uint32_t epoch,
                        const uint32_t* epoch_dev, uint32_t gen0, int n_gens, float* best_f, int* best_i,
                        int64_t* launches) {
    if (c->n_inst == 0) return METADE_OK;
    if (c->path == METADE_PATH_PLAIN || n_gens == 0) {
        // the grid barriers of this call's launches count up from zero
        if (n_gens > 0) CK(cudaMemsetAsync(c->bar, 0, sizeof(unsigned), st));
        unsigned base = 0;
        for (int g = 0; g < n_gens; ++g) {
            StepArgs a = step_args(c, pop, fit, theta, epoch, epoch_dev, gen0 + (uint32_t)g, 1, nullptr, nullptr);
            for (int k = 0; k < c->n_inst; ++k) {
                const unsigned nb = (unsigned)((c->hdesc[k].np + 7) / 8);
                if (base > 0xFFFFFFFFu - 2 * nb) {  // restart the count before it wraps
                    CK(cudaMemsetAsync(c->bar, 0, sizeof(unsigned), st));
                    base = 0;
                }
                CK(launch_plain_generation(a, k, c->hdesc[k], c->uscr, c->fuscr, c->topk, c->bar, base, st));
                base += 2 * nb;
                *launches += 1;
            }
        }
        if (best_f || best_i) {
            CK(launch_best(c->desc, c->n_inst, fit, best_f, best_i, st));
            *launches += 1;
        }
        return METADE_OK;
    }
    StepArgs a = step_args(c, pop, fit, theta, epoch, epoch_dev, gen0, n_gens, best_f, best_i);
    // The work of one call falls into independent units: each size bucket (one launch for all its
    // generations), the tensor-core pipeline and the MLP pipeline (launches per generation).  They
    // touch disjoint executors and scratch rows, so with more than one unit the buckets and the MLP
    // pipeline run on forked streams beside the tensor-core pipeline on `st` (inside a capture:
    // parallel branches of the graph), and `st` waits for all of them before the best reduction.
    const int units = (int)c->buckets.size() + (c->tc ? 1 : 0) + (c->mlpp.n_rows > 0 ? 1 : 0);
    int nside = 0;  // side streams forked so far
    auto unit_stream = [&](int q, cudaStream_t* out) -> cudaError_t {  // the q-th unit placed beside `st`
        *out = st;  // (st may be the legacy stream, 0)
        if (units <= 1) return cudaSuccess;
        const int sq = q % metade_ctx::kSide;
        if (sq >= nside) {
            cudaError_t e = nside == 0 ? cudaEventRecord(c->fork_ev, st) : cudaSuccess;
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side[sq], c->fork_ev, 0);
            if (e != cudaSuccess) return e;
            nside = sq + 1;
        }
        *out = c->side[sq];
        return cudaSuccess;
    };
    int q_unit = 0;
    for (const Bucket& b : c->buckets) {
        cudaStream_t bs;
        CK(unit_stream(q_unit++, &bs));
        cudaEvent_t e0, e1;
        const bool pr = prof_pair(c, bs,
                                  b.plan.kind == 0   ? kProfFusedSmall
                                  : b.plan.kind == 3 ? (b.plan.rot_smem ? kProfFusedTile : kProfFusedTileStream)
                                                     : kProfFusedGeneral,
                                  &e0, &e1);
        if (pr) cudaEventRecord(e0, bs);
        CK(launch_fused(a, c->work + b.work_off, b.n_work, b.plan, c->uscr, bs));
        if (pr) cudaEventRecord(e1, bs);
        *launches += 1;
    }
    if (c->tc) {
        for (int g = 0; g < n_gens; ++g) {
            StepArgs t = step_args(c, pop, fit, theta, epoch, epoch_dev, gen0 + (uint32_t)g, 1, nullptr, nullptr);
            cudaEvent_t ev[6];
            const bool sampled = !c->prof_on || c->prof_gen++ % c->prof_stride == 0;
            const bool pe = sampled && prof_tc(c, st, ev, c->tcp.fused != 0);
            if (c->tcp.fused) {
                CK(launch_tc_fused_generation(t, c->tcp, st, pe ? ev : nullptr));
                *launches += 4;
                continue;
            }
            CK(launch_tc_generation(t, c->tcp, st, pe ? ev : nullptr));
            *launches += 5;
        }
    }
    if (c->mlpp.n_rows > 0) {  // MLP executors: four launches per generation
        cudaStream_t ms = st;
        if (c->tc) CK(unit_stream(q_unit++, &ms));
        cudaEvent_t e0, e1;
        const bool pr = prof_pair(c, ms, kProfFusedMlp, &e0, &e1);
        if (pr) cudaEventRecord(e0, ms);
        for (int g = 0; g < n_gens; ++g) {
            StepArgs t = step_args(c, pop, fit, theta, epoch, epoch_dev, gen0 + (uint32_t)g, 1, nullptr, nullptr);
            CK(launch_mlp_generation(t, c->mlpp, ms));
            *launches += 4;
        }
        if (pr) cudaEventRecord(e1, ms);
    }
    for (int sq = 0; sq < nside; ++sq) {  // join
        CK(cudaEventRecord(c->join_ev[sq], c->side[sq]));
        CK(cudaStreamWaitEvent(st, c->join_ev[sq], 0));
    }
    // the per-generation paths leave best_f / best_i to one reduction over
    // every executor (the fused kernels write their own too)
    if ((c->tc || c->mlpp.n_rows > 0) && (best_f || best_i)) {
        CK(launch_best(c->desc, c->n_inst, fit, best_f, best_i, st));
        *launches += 1;
    }
    return METADE_OK;
}

metade_status run_init(metade_ctx* c, cudaStream_t st, float* pop, float* fit, uint32_t epoch,
                       const uint32_t* epoch_dev, int64_t* launches) {
    if (c->n_inst == 0) return METADE_OK;
    CK(launch_init(c->desc, c->n_inst, c->max_np, c->max_dpad, pop, make_key(c->seed, kTagInner), epoch, epoch_dev,
                   c->lo, c->hi, st));
    // executors on the tensor cores are evaluated by the rotation GEMM in the
    // context's precision, like every later evaluation of theirs
    // and the MLP objective's by its own evaluation kernel
    CK(launch_eval(c->desc, c->row_inst, c->n_indiv, pop, c->rotT, c->shift, false, fit, true, c->max_dpad, st,
                   c->tc || c->mlpp.n_rows > 0, c->mlp_x, c->mlp_y));
    *launches += 2;
    if (c->mlpp.n_rows > 0) {
        CK(launch_mlp_eval(c->desc, c->mlpp, pop, fit, c->status, st));
        *launches += 1;
    }
    if (c->tc) {
        CK(launch_tc_eval(c->desc, c->tcp, pop, c->shift, c->rotT, fit, c->status, st));
        *launches += 2;
    }
    return METADE_OK;
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

// Phase 0 of the context's evolver: the vectors to evaluate, decoded into theta.
cudaError_t launch_evolver_phase0(const metade_ctx* c, Key ko, const uint32_t* gen_dev, uint32_t gen, float* opop,
                                  float* ofit, float* trial, float* theta, cudaStream_t st) {
    switch (c->evolver) {
    case 1: return launch_pso_move(c->n_groups, c->n_out, ko, gen_dev, gen, opop, ofit, trial, theta, st);
    case 2: return launch_cso_move(c->n_groups, c->n_out, ko, gen_dev, gen, opop, ofit, trial, theta, st);
    case 3: return launch_nes_sample(c->n_groups, c->n_out, ko, gen_dev, gen, trial, theta, st);
    default: return launch_outer_trial(c->n_groups, c->n_out, ko, gen_dev, gen, opop, trial, theta, st);
    }
}

// Phase 1: the evolver's update from the meta-fitness of phase 0's vectors.
cudaError_t launch_evolver_phase1(const metade_ctx* c, float* opop, float* ofit, float* trial, const float* meta_fit,
                                  cudaStream_t st) {
    switch (c->evolver) {
    case 1: return launch_outer_select(c->n_groups, c->n_out, opop, ofit, trial, meta_fit, 12, st);
    case 2: return launch_cso_select(c->n_groups, c->n_out, opop, ofit, trial, meta_fit, st);
    case 3: return launch_nes_update(c->n_groups, c->n_out, opop, ofit, trial, meta_fit, st);
    default: return launch_outer_select(c->n_groups, c->n_out, opop, ofit, trial, meta_fit, 6, st);
    }
}

// The evolver generation as a stream sequence (captured into a graph or run directly).
metade_status enqueue_outer_generation(metade_ctx* c, cudaStream_t st, float* opop, float* ofit, float* trial,
                                       float* theta, float* pop, float* fit, float* best_f, int* best_i,
                                       int n_inner, int64_t* launches) {
    const Key ko = make_key(c->seed, kTagOuter);
    CK(launch_evolver_phase0(c, ko, c->gen_dev, 0, opop, ofit, trial, theta, st));
    *launches += 1;
    const uint32_t* ep = c->one_shot ? nullptr : c->gen_dev;
    metade_status s = run_init(c, st, pop, fit, 0, ep, launches);
    if (s != METADE_OK) return s;
    s = run_inner(c, st, pop, fit, theta, 0, ep, 0, n_inner, best_f, best_i, launches);
    if (s != METADE_OK) return s;
    CK(launch_evolver_phase1(c, opop, ofit, trial, best_f, st));
    *launches += 1;
    return METADE_OK;
}

}  // namespace

extern "C" {

const char* metade_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda); }

const char* metade_strerror(metade_status s) {
    switch (s) {
    case METADE_OK: return "ok";
    case METADE_EINVAL: return "invalid argument";
    case METADE_ENOMEM: return "out of device memory";
    case METADE_ECUDA: return "CUDA error";
    case METADE_ETIMEOUT: return "device wait timed out";
    case METADE_ESTATE: return "call not valid in this state";
    case METADE_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

void metade_destroy(metade_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    cudaFree(c->desc);
    cudaFree(c->row_inst);
    cudaFree(c->rot);
    cudaFree(c->rotT);
    cudaFree(c->shift);
    cudaFree(c->uscr);
    cudaFree(c->fuscr);
    cudaFree(c->topk);
    cudaFree(c->status);
    cudaFree(c->gen_dev);
    cudaFree(c->bar);
    cudaFree(c->work);
    free_tc(c);
    cudaFree(c->tie_total);
    cudaFree(c->mlp_x);
    cudaFree(c->mlp_y);
    cudaFree(c->mlp_execs);
    cudaFree(c->mlp_row_exec);
    cudaFree(c->mlp_topk);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int q = 0; q < metade_ctx::kSide; ++q) {
        if (c->side[q]) cudaStreamDestroy(c->side[q]);
        if (c->join_ev[q]) cudaEventDestroy(c->join_ev[q]);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    delete c;
}

metade_status metade_create(const metade_config* cfg, metade_ctx** out) {
    if (!out) return METADE_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->n_prob < 1 || cfg->n_inst < 0 || !cfg->prob_dim || !cfg->prob_obj) return METADE_EINVAL;
    if (cfg->n_inst > 0 && (!cfg->inst_np || !cfg->inst_prob || !cfg->shift || !cfg->rot)) return METADE_EINVAL;
    if (!(cfg->lo < cfg->hi) || !std::isfinite(cfg->lo) || !std::isfinite(cfg->hi)) return METADE_EINVAL;
    if (cfg->p_best_pct < 0 || cfg->p_best_pct > 100) return METADE_EINVAL;
    if (cfg->n_out < 0 || (cfg->n_out > 0 && (cfg->n_out < 4 || cfg->n_inst % cfg->n_out != 0))) return METADE_EINVAL;
    if (cfg->path != METADE_PATH_BATCHED && cfg->path != METADE_PATH_PLAIN) return METADE_EINVAL;
    if (cfg->prec != METADE_FP32 && cfg->prec != METADE_BF16 && cfg->prec != METADE_BF16X3 &&
        cfg->prec != METADE_FP8E4M3)
        return METADE_EUNSUPPORTED;
    for (int p = 0; p < cfg->n_prob; ++p) {
        if (cfg->prob_dim[p] < 1 || cfg->prob_obj[p] < 0 || cfg->prob_obj[p] > kMlp) return METADE_EINVAL;
        if (cfg->prob_obj[p] == kMlp) {
            if (!mlp_hidden(cfg->prob_dim[p])) return METADE_EINVAL;      // D = 19 h + 2
            if (cfg->path == METADE_PATH_PLAIN) return METADE_EUNSUPPORTED;  // batched kernel only
        }
        if (cfg->prob_dim[p] > kMaxDim) return METADE_EUNSUPPORTED;
    }
    for (int k = 0; k < cfg->n_inst; ++k) {
        if (cfg->inst_np[k] < 4 || cfg->inst_np[k] > kMaxNp) return METADE_EINVAL;
        if (cfg->inst_prob[k] < 0 || cfg->inst_prob[k] >= cfg->n_prob) return METADE_EINVAL;
        if (cfg->inst_group && cfg->inst_group[k] < 0) return METADE_EINVAL;
    }

    if (cfg->evolver < 0 || cfg->evolver > 3) return METADE_EINVAL;
    if (cfg->tc_min_dim < 0) return METADE_EINVAL;
    if (cfg->evolver == 2 && cfg->n_out > 4096) return METADE_EINVAL;  // the pairing lives in shared memory

    metade_ctx* c = new metade_ctx();
    c->n_prob = cfg->n_prob;
    c->n_inst = cfg->n_inst;
    c->n_out = cfg->n_out;
    c->n_groups = cfg->n_out > 0 ? cfg->n_inst / cfg->n_out : 0;
    c->lo = cfg->lo;
    c->hi = cfg->hi;
    c->seed = cfg->seed;
    c->one_shot = cfg->one_shot ? 1 : 0;
    c->p_best_pct = cfg->p_best_pct == 0 ? 10 : cfg->p_best_pct;
    c->prec = cfg->prec;
    c->path = cfg->path;
    c->tie_fp64 = cfg->tie_fp64 ? 1 : 0;
    c->evolver = cfg->evolver;
    c->st = (cudaStream_t)cfg->stream;

    // problem tables: input offsets (unpadded) and padded offsets
    std::vector<long long> rot_in_off(c->n_prob), rot_off(c->n_prob);
    std::vector<int> shift_in_off(c->n_prob), shift_off(c->n_prob);
    std::vector<int> mlp_yoff(c->n_prob, 0);  // MLP problems: offset of their targets
    int n_mlp = 0;
    long long rin = 0, rpad = 0;
    int sin_ = 0, spad = 0;
    for (int p = 0; p < c->n_prob; ++p) {
        const int D = cfg->prob_dim[p], Dp = (D + 3) & ~3;
        rot_in_off[p] = rin;
        rot_off[p] = rpad;
        shift_in_off[p] = sin_;
        shift_off[p] = spad;
        rin += (long long)D * D;
        rpad += (long long)D * Dp;
        sin_ += D;
        spad += Dp;
        c->max_dim = std::max(c->max_dim, D);
        if (cfg->prob_obj[p] == kMlp) mlp_yoff[p] = kMlpN * kMlpOut * n_mlp++;
    }

    c->hdesc.resize(c->n_inst);
    c->pop_off.resize(c->n_inst);
    c->fit_off.resize(c->n_inst);
    c->dpad.resize(c->n_inst);
    std::vector<int> row_inst;
    long long po = 0, fo = 0;
    for (int k = 0; k < c->n_inst; ++k) {
        const int p = cfg->inst_prob[k];
        const int D = cfg->prob_dim[p], Dp = (D + 3) & ~3, np = cfg->inst_np[k];
        InstDesc d;
        std::memset(&d, 0, sizeof(d));
        d.pop_off = po;
        d.rot_off = rot_off[p];
        d.fit_off = (int)fo;
        d.np = np;
        d.dim = D;
        d.dpad = Dp;
        d.obj = cfg->prob_obj[p];
        const int group = cfg->inst_group ? cfg->inst_group[k] : (c->n_out > 0 ? k / c->n_out : 0);
        d.stream = c->one_shot ? group : k;
        d.shift_off = shift_off[p];
        d.kp = std::max(1, (np * c->p_best_pct + 99) / 100);
        d.prob = p;
        d.aux = mlp_yoff[p];
        c->hdesc[k] = d;
        c->pop_off[k] = po;
        c->fit_off[k] = fo;
        c->dpad[k] = Dp;
        for (int i = 0; i < np; ++i) row_inst.push_back(k);
        po += (long long)np * Dp;
        fo += np;
        c->max_np = std::max(c->max_np, np);
        c->max_dpad = std::max(c->max_dpad, Dp);
        c->max_kp = std::max(c->max_kp, d.kp);
    }
    if (fo >= (1LL << 31)) {
        delete c;
        return METADE_EUNSUPPORTED;
    }
    // executors of the MLP objective: their first row (InstDesc.tc_row) in the MLP row list
    std::vector<int> mlp_execs, mlp_row_exec;
    for (int k = 0; k < c->n_inst; ++k) {
        InstDesc& d = c->hdesc[k];
        if (d.obj != kMlp) continue;
        d.tc_row = (int)mlp_row_exec.size();
        mlp_execs.push_back(k);
        for (int i = 0; i < d.np; ++i) mlp_row_exec.push_back(k);
    }
    c->pop_floats = po;
    c->n_indiv = fo;

    auto fail = [&](metade_status s) {
        metade_destroy(c);
        return s;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(METADE_ECUDA);
    e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    for (int q = 0; q < metade_ctx::kSide && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&c->side[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev[q], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(METADE_ECUDA);
    if (dalloc(&c->desc, c->n_inst) || dalloc(&c->row_inst, row_inst.size()) || dalloc(&c->rot, rpad) ||
        dalloc(&c->rotT, rpad) || dalloc(&c->shift, spad) || dalloc(&c->uscr, po) || dalloc(&c->fuscr, fo) ||
        dalloc(&c->topk, c->max_np) || dalloc(&c->status, 1) || dalloc(&c->gen_dev, 1) || dalloc(&c->bar, 1))
        return fail(METADE_ENOMEM);
    if (cudaMemset(c->status, 0, sizeof(int)) || cudaMemset(c->gen_dev, 0, sizeof(uint32_t)) ||
        cudaMemset(c->uscr, 0, sizeof(float) * (size_t)std::max(po, 1LL)))
        return fail(METADE_ECUDA);
    if (c->n_inst > 0) {
        if (cudaMemcpy(c->desc, c->hdesc.data(), sizeof(InstDesc) * c->n_inst, cudaMemcpyHostToDevice) ||
            cudaMemcpy(c->row_inst, row_inst.data(), sizeof(int) * row_inst.size(), cudaMemcpyHostToDevice))
            return fail(METADE_ECUDA);
        // pad the problem table on the device
        long long* d_rio = nullptr;
        long long* d_ro = nullptr;
        int *d_sio = nullptr, *d_so = nullptr, *d_dim = nullptr;
        std::vector<int> dims(cfg->prob_dim, cfg->prob_dim + c->n_prob);
        bool ok = !dalloc(&d_rio, c->n_prob) && !dalloc(&d_ro, c->n_prob) && !dalloc(&d_sio, c->n_prob) &&
                  !dalloc(&d_so, c->n_prob) && !dalloc(&d_dim, c->n_prob);
        ok = ok && !cudaMemcpy(d_rio, rot_in_off.data(), sizeof(long long) * c->n_prob, cudaMemcpyHostToDevice) &&
             !cudaMemcpy(d_ro, rot_off.data(), sizeof(long long) * c->n_prob, cudaMemcpyHostToDevice) &&
             !cudaMemcpy(d_sio, shift_in_off.data(), sizeof(int) * c->n_prob, cudaMemcpyHostToDevice) &&
             !cudaMemcpy(d_so, shift_off.data(), sizeof(int) * c->n_prob, cudaMemcpyHostToDevice) &&
             !cudaMemcpy(d_dim, dims.data(), sizeof(int) * c->n_prob, cudaMemcpyHostToDevice);
        ok = ok && !launch_pad_problems(cfg->rot, cfg->shift, d_rio, d_sio, d_dim, d_ro, d_so, c->n_prob, c->max_dim,
                                        c->rot, c->rotT, c->shift, c->st);
        ok = ok && !cudaStreamSynchronize(c->st);
        cudaFree(d_rio);
        cudaFree(d_ro);
        cudaFree(d_sio);
        cudaFree(d_so);
        cudaFree(d_dim);
        if (!ok) return fail(METADE_ECUDA);
        c->launches += 1;
        if (n_mlp > 0) {  // MLP objective: the fixed inputs and every problem's teacher outputs
            if (dalloc(&c->mlp_x, (size_t)kMlpN * kMlpIn) || dalloc(&c->mlp_y, (size_t)kMlpN * kMlpOut * n_mlp))
                return fail(METADE_ENOMEM);
            bool okm = !launch_mlp_inputs(c->mlp_x, c->st);
            for (int p = 0; p < c->n_prob && okm; ++p)
                if (cfg->prob_obj[p] == kMlp)
                    okm = !launch_mlp_targets(c->mlp_x, c->shift + shift_off[p], mlp_hidden(cfg->prob_dim[p]),
                                              c->mlp_y + mlp_yoff[p], c->st);
            if (!okm || cudaStreamSynchronize(c->st)) return fail(METADE_ECUDA);
            c->launches += 1 + n_mlp;
            if (dalloc(&c->mlp_execs, mlp_execs.size()) || dalloc(&c->mlp_row_exec, mlp_row_exec.size()) ||
                dalloc(&c->mlp_topk, (size_t)c->n_indiv))
                return fail(METADE_ENOMEM);
            if (cudaMemcpy(c->mlp_execs, mlp_execs.data(), sizeof(int) * mlp_execs.size(), cudaMemcpyHostToDevice) ||
                cudaMemcpy(c->mlp_row_exec, mlp_row_exec.data(), sizeof(int) * mlp_row_exec.size(),
                           cudaMemcpyHostToDevice))
                return fail(METADE_ECUDA);
            MlpPlan& m = c->mlpp;
            m.execs = c->mlp_execs;
            m.n_exec = (int)mlp_execs.size();
            m.row_exec = c->mlp_row_exec;
            m.n_rows = (int)mlp_row_exec.size();
            m.topk_all = c->mlp_topk;
            m.uscr = c->uscr;
            m.fu = c->fuscr;
            m.x = c->mlp_x;
            m.y = c->mlp_y;
            m.max_dpad = 0;
            for (int k : mlp_execs) m.max_dpad = std::max(m.max_dpad, c->hdesc[k].dpad);
            // BF16 / bf16x3 contexts evaluate the first layer on the tensor cores; FP32 and FP8 on the CUDA cores
            m.tc = c->prec == METADE_BF16 ? 1 : c->prec == METADE_BF16X3 ? 2 : 0;
            m.sms = std::max(1, device_sms());
            if ((size_t)8 * m.max_dpad * sizeof(float) > kSmemLimit) return fail(METADE_EUNSUPPORTED);
        }
    }
    c->tc_unfused = cfg->tc_unfused ? 1 : 0;
    c->tc_auto = cfg->tc_min_dim == 0;
    c->tc_min_dim = cfg->tc_min_dim > 0 ? cfg->tc_min_dim
                    : (c->prec == METADE_FP32 ? kSimtDefaultMinDim : kTcDefaultMinDim);
    if (c->n_inst > 0) {
        metade_status s = setup_tc(c);
        if (s == METADE_OK) s = build_plan(c);
        if (s != METADE_OK) return fail(s);
    }
    *out = c;
    return METADE_OK;
}

metade_status metade_layout(const metade_ctx* c, int64_t* pop_floats, int64_t* n_indiv, int32_t* n_groups) {
    if (!c) return METADE_EINVAL;
    if (pop_floats) *pop_floats = c->pop_floats;
    if (n_indiv) *n_indiv = c->n_indiv;
    if (n_groups) *n_groups = c->n_groups;
    return METADE_OK;
}

metade_status metade_offsets(const metade_ctx* c, int64_t* pop_off, int64_t* fit_off, int32_t* dpad) {
    if (!c) return METADE_EINVAL;
    for (int k = 0; k < c->n_inst; ++k) {
        if (pop_off) pop_off[k] = c->pop_off[k];
        if (fit_off) fit_off[k] = c->fit_off[k];
        if (dpad) dpad[k] = c->dpad[k];
    }
    return METADE_OK;
}

metade_status metade_set_stream(metade_ctx* c, void* stream) {
    if (!c) return METADE_EINVAL;
    c->st = (cudaStream_t)stream;
    return METADE_OK;
}

metade_status metade_init(metade_ctx* c, float* pop, float* fit, uint32_t epoch) {
    if (!c || (c->n_inst > 0 && (!pop || !fit))) return METADE_EINVAL;
    if (epoch > 0xFFFFu) return METADE_EINVAL;
    return run_init(c, c->st, pop, fit, epoch, nullptr, &c->launches);
}

metade_status metade_inner_step(metade_ctx* c, float* pop, float* fit, const float* theta, uint32_t epoch,
                                uint32_t gen0, int32_t n_gens, float* best_f, int32_t* best_i) {
    if (!c || n_gens < 0 || epoch > 0xFFFFu) return METADE_EINVAL;
    if (c->n_inst > 0 && (!pop || !fit || !theta)) return METADE_EINVAL;
    return run_inner(c, c->st, pop, fit, theta, epoch, nullptr, gen0, n_gens, best_f, best_i, &c->launches);
}

metade_status metade_eval(metade_ctx* c, const float* x, int64_t n, const int32_t* inst, int32_t ldx,
                          metade_prec prec, void* f_out) {
    if (!c || n < 0) return METADE_EINVAL;
    if (prec != METADE_FP32 && prec != METADE_FP64) return METADE_EUNSUPPORTED;
    if (n == 0) return METADE_OK;
    if (!x || !inst || !f_out || ldx < 4 || (ldx & 3) || ((uintptr_t)x & 15)) return METADE_EINVAL;
    if (c->n_inst == 0) return METADE_EINVAL;  // no executor a point could belong to
    CK(launch_eval(c->desc, nullptr, n, x, c->rotT, c->shift, prec == METADE_FP64, f_out, false, c->max_dpad, c->st,
                   false, c->mlp_x, c->mlp_y, inst, ldx, c->n_inst, c->status));
    c->launches += 1;
    return METADE_OK;
}

metade_status metade_eval_pop(metade_ctx* c, const float* pop, metade_prec prec, void* f_out) {
    if (!c || (c->n_inst > 0 && (!pop || !f_out))) return METADE_EINVAL;
    if (prec != METADE_FP32 && prec != METADE_FP64) return METADE_EUNSUPPORTED;
    if (c->n_inst == 0) return METADE_OK;
    CK(launch_eval(c->desc, c->row_inst, c->n_indiv, pop, c->rotT, c->shift, prec == METADE_FP64, f_out, false,
                   c->max_dpad, c->st, false, c->mlp_x, c->mlp_y));
    c->launches += 1;
    return METADE_OK;
}

metade_status metade_outer_init(metade_ctx* c, float* opop, float* ofit) {
    if (!c) return METADE_EINVAL;
    if (c->n_out == 0) return METADE_ESTATE;
    if (!opop || !ofit) return METADE_EINVAL;
    CK(launch_outer_init(c->n_groups, c->n_out, make_key(c->seed, kTagOuter), opop, ofit, c->st));
    c->launches += 1;
    return METADE_OK;
}

metade_status metade_outer_step(metade_ctx* c, float* opop, float* ofit, float* trial, float* theta,
                                const float* meta_fit, uint32_t outer_gen, int32_t phase) {
    if (!c) return METADE_EINVAL;
    if (c->n_out == 0) return METADE_ESTATE;
    if (phase == 0) {
        if (!opop || !trial || !theta || ((c->evolver == 1 || c->evolver == 2) && !ofit)) return METADE_EINVAL;
        CK(launch_evolver_phase0(c, make_key(c->seed, kTagOuter), nullptr, outer_gen, opop, ofit, trial, theta, c->st));
    } else if (phase == 1) {
        if (!opop || !ofit || !trial || !meta_fit) return METADE_EINVAL;
        CK(launch_evolver_phase1(c, opop, ofit, trial, meta_fit, c->st));
    } else {
        return METADE_EINVAL;
    }
    c->launches += 1;
    return METADE_OK;
}

metade_status metade_outer_generation(metade_ctx* c, float* opop, float* ofit, float* trial, float* theta,
                                      float* pop, float* fit, float* best_f, int32_t* best_i, uint32_t outer_gen,
                                      int32_t n_inner, int32_t use_graph) {
    if (!c) return METADE_EINVAL;
    if (c->n_out == 0) return METADE_ESTATE;
    if (!opop || !ofit || !trial || !theta || !pop || !fit || !best_f || n_inner < 0 || outer_gen > 0xFFFFu)
        return METADE_EINVAL;
    k_set_u32<<<1, 1, 0, c->st>>>(c->gen_dev, outer_gen);
    CK(cudaGetLastError());
    c->launches += 1;
    // the plain path is the no-graph baseline: always launched directly
    if (!use_graph || c->path == METADE_PATH_PLAIN)
        return enqueue_outer_generation(c, c->st, opop, ofit, trial, theta, pop, fit, best_f, best_i, n_inner,
                                        &c->launches);
    std::vector<uintptr_t> key = {(uintptr_t)opop, (uintptr_t)ofit, (uintptr_t)trial, (uintptr_t)theta,
                                  (uintptr_t)pop, (uintptr_t)fit, (uintptr_t)best_f, (uintptr_t)best_i,
                                  (uintptr_t)n_inner};
    GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
        if (g.key == key) ge = &g;
    if (!ge) {
        // capture on the private stream, ordered after the caller's stream
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, c->st));
        CK(cudaStreamWaitEvent(c->cap, ev, 0));
        CK(cudaStreamSynchronize(c->cap));
        cudaEventDestroy(ev);
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        int64_t kernels = 0;
        metade_status s =
            enqueue_outer_generation(c, c->cap, opop, ofit, trial, theta, pop, fit, best_f, best_i, n_inner, &kernels);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
        if (s != METADE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        CK(e);
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        c->graphs.push_back(GraphEntry{key, exec, kernels});
        ge = &c->graphs.back();
    }
    CK(cudaGraphLaunch(ge->exec, c->st));
    c->launches += ge->kernels;
    return METADE_OK;
}

metade_status metade_draw_record(metade_ctx* c, const float* fit, const float* theta, uint32_t epoch, uint32_t gen,
                                 int32_t* rec) {
    if (!c || epoch > 0xFFFFu) return METADE_EINVAL;
    if (c->n_inst == 0) return METADE_OK;
    if (!fit || !theta || !rec) return METADE_EINVAL;
    StepArgs a = step_args(c, nullptr, const_cast<float*>(fit), theta, epoch, nullptr, gen, 1, nullptr, nullptr);
    CK(launch_record(a, c->n_inst, c->max_np, rec, c->st));
    c->launches += 1;
    return METADE_OK;
}

metade_status metade_sync(metade_ctx* c) {
    if (!c) return METADE_EINVAL;
    CK(cudaStreamSynchronize(c->st));
    int s = 0;
    CK(cudaMemcpy(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (s != 0) CK(cudaMemset(c->status, 0, sizeof(int)));
    return (metade_status)s;
}

metade_status metade_autotune(metade_ctx* c, const float* pop, const float* fit, const float* theta, int32_t n_gens) {
    if (!c || n_gens < 1 || (c->n_inst > 0 && (!pop || !fit || !theta))) return METADE_EINVAL;
    if (c->path != METADE_PATH_BATCHED || c->n_inst == 0) return METADE_OK;
    const bool fp32 = c->prec == METADE_FP32;
    const int alt_w = fp32 ? kSimtDefaultMinDim : kTcAltMinDim;
    bool mid = false;  // executors whose place (per-generation GEMM pipeline or fused kernels) the width decides
    for (const InstDesc& d : c->hdesc)
        mid = mid || (d.obj != kMlp && d.dim >= kTcLowMinDim && d.dim < alt_w);
    const bool tune_width = c->tc_auto && mid;
    if (c->buckets.empty() && !tune_width) return METADE_OK;
    // the plan changes: graphs captured with the old one are dropped
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    float* tpop = nullptr;
    float* tfit = nullptr;
    if (dalloc(&tpop, (size_t)c->pop_floats) || dalloc(&tfit, (size_t)c->n_indiv)) {
        cudaFree(tpop);
        return METADE_ENOMEM;
    }
    cudaEvent_t e0, e1;
    metade_status st = METADE_OK;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) st = METADE_ECUDA;
    if (st == METADE_OK && tune_width) {
        // the tensor-core width: n_gens whole generations of every executor per candidate
        const bool prof = c->prof_on;
        c->prof_on = false;
        int best_w = c->tc_min_dim;
        float best_ms = -1.f;
        c->tc_tuned.clear();
        for (int w : {kTcLowMinDim, kTcDefaultMinDim, alt_w}) {
            c->tc_min_dim = w;
            st = setup_tc(c);
            if (st == METADE_OK) st = build_plan(c);
            if (st != METADE_OK) break;
            int64_t nl = 0;
            // one untimed generation first: the first launch of a kernel also loads it
            if (cudaMemcpyAsync(tpop, pop, sizeof(float) * (size_t)c->pop_floats, cudaMemcpyDeviceToDevice, c->st) ||
                cudaMemcpyAsync(tfit, fit, sizeof(float) * (size_t)c->n_indiv, cudaMemcpyDeviceToDevice, c->st)) {
                st = METADE_ECUDA;
                break;
            }
            st = run_inner(c, c->st, tpop, tfit, theta, 0, nullptr, 0, 1, nullptr, nullptr, &nl);
            if (st != METADE_OK) break;
            if (cudaMemcpyAsync(tpop, pop, sizeof(float) * (size_t)c->pop_floats, cudaMemcpyDeviceToDevice, c->st) ||
                cudaMemcpyAsync(tfit, fit, sizeof(float) * (size_t)c->n_indiv, cudaMemcpyDeviceToDevice, c->st) ||
                cudaEventRecord(e0, c->st)) {
                st = METADE_ECUDA;
                break;
            }
            st = run_inner(c, c->st, tpop, tfit, theta, 0, nullptr, 0, n_gens, nullptr, nullptr, &nl);
            if (st != METADE_OK) break;
            if (cudaEventRecord(e1, c->st) || cudaEventSynchronize(e1)) {
                st = METADE_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            char tmp[64];
            snprintf(tmp, sizeof(tmp), "%s\"%d\": %.4f", c->tc_tuned.empty() ? "" : ", ", w, ms);
            c->tc_tuned += tmp;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                best_w = w;
            }
        }
        c->prof_on = prof;
        c->tc_min_dim = best_w;
        if (st == METADE_OK) st = setup_tc(c);
        if (st == METADE_OK) st = build_plan(c);
    }
    for (Bucket& b : c->buckets) {
        if (st != METADE_OK) break;
        std::vector<int> cands = b.plan.kind == 0 ? std::vector<int>{32, 64, 128, 256}
                                                  : std::vector<int>{128, 256, 512};
        if (b.plan.kind == 3) cands = b.plan.rot_smem ? std::vector<int>{128, 256} : std::vector<int>{256};
        FusedPlan best = b.plan;
        float best_ms = -1.f;
        b.tuned.clear();
        for (int th : cands) {
            FusedPlan p = b.plan;
            p.threads = th;
            if (p.kind == 1) {
                p.rot_smem = fused_smem_general(p.max_np, p.max_dpad, th, true) <= kSmemLimit ? 1 : 0;
                p.smem = fused_smem_general(p.max_np, p.max_dpad, th, p.rot_smem != 0);
                if (p.smem > kSmemLimit) continue;
            } else if (p.kind == 3) {
                p.smem = fused_smem_tile(p.max_np, p.max_dpad, th, p.rot_smem != 0);
                if (p.smem > kSmemLimit) continue;
            } else if (th < 32) {
                continue;
            }
            StepArgs a = step_args(c, tpop, tfit, theta, 0, nullptr, 0, n_gens, nullptr, nullptr);
            if (cudaMemcpyAsync(tpop, pop, sizeof(float) * (size_t)c->pop_floats, cudaMemcpyDeviceToDevice, c->st) ||
                cudaMemcpyAsync(tfit, fit, sizeof(float) * (size_t)c->n_indiv, cudaMemcpyDeviceToDevice, c->st) ||
                cudaEventRecord(e0, c->st) || launch_fused(a, c->work + b.work_off, b.n_work, p, c->uscr, c->st) ||
                cudaEventRecord(e1, c->st) || cudaEventSynchronize(e1)) {
                st = METADE_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            char tmp[64];
            snprintf(tmp, sizeof(tmp), "%s\"%d\": %.4f", b.tuned.empty() ? "" : ", ", th, ms);
            b.tuned += tmp;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                best = p;
            }
        }
        b.plan = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tpop);
    cudaFree(tfit);
    if (st == METADE_OK && cudaMemset(c->status, 0, sizeof(int))) st = METADE_ECUDA;
    return st;
}

metade_status metade_plan_info(const metade_ctx* c, char* buf, size_t len) {
    if (!c || !buf || len == 0) return METADE_EINVAL;
    std::string s = "{\"path\": \"";
    s += c->path == METADE_PATH_PLAIN ? "plain" : "batched";
    s += "\", \"buckets\": [";
    for (size_t b = 0; b < c->buckets.size(); ++b) {
        const Bucket& k = c->buckets[b];
        char tmp[256];
        snprintf(tmp, sizeof(tmp),
                 "%s{\"kernel\": \"%s\", \"dmax\": %d, \"threads\": %d, \"grid\": %d, \"smem\": %zu, "
                 "\"rot_smem\": %d, \"pop_smem\": %d, \"executors\": %d",
                 b ? ", " : "",
                 k.plan.kind == 0   ? "fused_small"
                 : k.plan.kind == 3 ? (k.plan.rot_smem ? "fused_tile" : "fused_tile_stream")
                                    : "fused_general",
                 k.plan.dmax,
                 k.plan.threads,
                 k.plan.grid, k.plan.smem, k.plan.rot_smem, k.plan.pop_smem, k.n_work);
        s += tmp;
        if (!k.tuned.empty()) s += ", \"autotune_ms\": {" + k.tuned + "}";
        s += "}";
    }
    s += "]";
    {
        char tmp[160];
        snprintf(tmp, sizeof(tmp), ", \"tc_min_dim\": %d, \"tc_min_dim_auto\": %s", c->tc_min_dim,
                 c->tc_auto ? "true" : "false");
        s += tmp;
        if (!c->tc_tuned.empty()) s += ", \"tc_autotune_ms\": {" + c->tc_tuned + "}";
    }
    if (c->tc) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp),
                 ", \"tensor_core\": {\"kernel\": \"%s\", \"precision\": \"%s\", \"executors\": %d, "
                 "\"tiles\": %d, \"kp\": %d, \"tile\": [%d, 256, %d], \"kernels_per_generation\": %d}",
                 c->tcp.simt ? "k_rot_simt" : c->tcp.fused == 1 ? "k_tc_sel" : "k_rot_tc",
                 c->tcp.simt ? "fp32" : c->tcp.fp8 ? "fp8e4m3" : c->tcp.split ? "bf16x3" : "bf16", c->tcp.n_exec,
                 c->tcp.n_tiles, c->tcp.kp, c->tcp.simt ? 64 : 128, c->tcp.simt ? 16 : 64, c->tcp.fused ? 4 : 5);
        s += tmp;
    }
    if (c->mlpp.n_rows > 0) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp),
                 ", \"mlp\": {\"kernels\": [\"k_mlp_prologue\", \"k_mlp_trial\", \"%s\", \"k_mlp_select\"], "
                 "\"precision\": \"%s\", \"executors\": %d, \"rows\": %d}",
                 c->mlpp.tc ? "k_mlp_tc" : "k_mlp_eval",
                 c->mlpp.tc == 1 ? "bf16" : c->mlpp.tc == 2 ? "bf16x3" : "fp32", c->mlpp.n_exec, c->mlpp.n_rows);
        s += tmp;
    }
    s += "}";
    if (s.size() + 1 > len) return METADE_EINVAL;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return METADE_OK;
}

int64_t metade_launch_count(const metade_ctx* c) { return c ? c->launches : -1; }

metade_status metade_profile(metade_ctx* c, int32_t enable) {
    if (!c || enable < 0) return METADE_EINVAL;
    c->prof_on = enable != 0;
    c->prof_stride = enable > 1 ? enable : 1;
    return METADE_OK;
}

metade_status metade_profile_read(metade_ctx* c, double* ms, int64_t* count) {
    if (!c) return METADE_EINVAL;
    CK(cudaStreamSynchronize(c->st));
    double tot[kProfKinds] = {};
    int64_t n[kProfKinds] = {};
    for (auto& r : c->prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            tot[r.kind] += t;
            n[r.kind] += 1;
        }
    }
    c->prof.clear();
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    c->prof_events.clear();
    if (c->tie_total) {
        unsigned long long h = 0;
        CK(cudaMemcpy(&h, c->tie_total, sizeof(h), cudaMemcpyDeviceToHost));
        CK(cudaMemset(c->tie_total, 0, sizeof(h)));
        n[kProfNearTies] = (int64_t)h;
    }
    for (int k = 0; k < kProfKinds; ++k) {
        if (ms) ms[k] = tot[k];
        if (count) count[k] = n[k];
    }
    return METADE_OK;
}

metade_status metade_wait_check(int32_t arrive, uint32_t rounds, int32_t* completed, double* seconds) {
    if (arrive != 0 && arrive != 1) return METADE_EINVAL;
    long long* d = nullptr;
    int* st = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(long long)) != cudaSuccess) return METADE_ENOMEM;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
        cudaFree(d);
        return METADE_ENOMEM;
    }
    long long h[2] = {0, 0};
    int hs = 0, khz = 0, dev = 0;
    metade_status r = METADE_OK;
    if (cudaMemset(d, 0, 2 * sizeof(long long)) || cudaMemset(st, 0, sizeof(int)) ||
        launch_wait_check(rounds, arrive, d, st, 0) || cudaDeviceSynchronize() ||
        cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) || cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost) ||
        cudaGetDevice(&dev) || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev))
        r = METADE_ECUDA;
    cudaFree(d);
    cudaFree(st);
    if (r != METADE_OK) return r;
    if (completed) *completed = (int32_t)h[0];
    if (seconds) *seconds = khz > 0 ? (double)h[1] / (1e3 * khz) : 0.0;
    return hs ? (metade_status)hs : METADE_OK;
}

}  // extern "C"
