// internal.h -- host-side launchers shared by the translation units of the
// library (not part of the C-ABI).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"

namespace metade {

struct StepArgs {
    const InstDesc* desc;
    float* pop;
    float* fit;
    const float* theta;
    const float* rot;    // padded R rows [dim][dpad] per problem
    const float* rotT;   // padded R^T [dim][dpad] per problem
    const float* shift;  // padded o [dpad] per problem
    Key key;
    uint32_t epoch, gen0;
    const uint32_t* epoch_dev;  // when non-null, the epoch is read here (graph replays)
    int n_gens;
    float lo, hi;
    float* best_f;
    int* best_i;
    int* status;
    int tie_fp64;  // 1: FP64 re-evaluation of both vectors; 0: FP32 difference form
};

// Problem table: pad R to rows of dpad floats, build R^T, pad o.
cudaError_t launch_pad_problems(const float* rot_in, const float* shift_in, const long long* rot_in_off,
                                const int* shift_in_off, const int* dims, const long long* rot_off,
                                const int* shift_off, int n_prob, int max_dim, float* rot, float* rotT,
                                float* shift, cudaStream_t st);

cudaError_t launch_init(const InstDesc* desc, int n_inst, int max_np, int max_dpad, float* pop, Key key,
                        uint32_t epoch, const uint32_t* epoch_dev, float lo, float hi, cudaStream_t st);

// Evaluate every row (row_inst maps rows to executors).  f64 selects FP64;
// skip_tc leaves the rows of executors on the tensor-core and MLP paths
// untouched (those paths evaluate them).  With pt_inst, n_rows caller-given
// points instead: point r at pop + r * ldx, executor pt_inst[r] (bad ids or
// dimensions above ldx latch EINVAL in *status and give NaN).
cudaError_t launch_eval(const InstDesc* desc, const int* row_inst, long long n_rows, const float* pop,
                        const float* rotT, const float* shift, bool f64, void* f_out, bool nan_inf,
                        int max_dpad, cudaStream_t st, bool skip_tc, const float* mlp_x = nullptr,
                        const float* mlp_y = nullptr, const int* pt_inst = nullptr, int ldx = 0, int n_inst = 0,
                        int* status = nullptr);

cudaError_t launch_record(const StepArgs& a, int n_inst, int max_np, int* rec, cudaStream_t st);

cudaError_t launch_best(const InstDesc* desc, int n_inst, const float* fit, float* best_f, int* best_i,
                        cudaStream_t st);

// Plain path: one executor, one generation, one cooperative launch
// (ceil(NP / 8) CTAs).  *bar counts grid-barrier arrivals from zero over the
// caller's sequence of launches; `base` is the count before this launch
// (each launch adds 2 ceil(NP / 8)).
cudaError_t launch_plain_generation(const StepArgs& a, int k, const InstDesc& d, float* u_scratch,
                                    float* fu_scratch, int* topk_scratch, unsigned* bar, unsigned base,
                                    cudaStream_t st);

// Batched path: executors listed in `work` (schedule order), all n_gens generations.
struct FusedPlan {
    int kind;      // 0 small (thread per individual), 1 general (warp per individual),
                   // 3 tile (register-blocked rotation GEMM per tile of individuals)
    int dmax;      // small: compile-time row bound
    int threads;   // block size
    int grid;      // CTAs (<= n_work; CTAs loop over work items)
    size_t smem;   // dynamic shared memory per CTA
    int rot_smem;  // general, tile: R^T staged in shared memory (tile: else streamed by chunks)
    int pop_smem;  // small: the population resident in shared memory for all fused generations
    int max_np, max_dpad;  // general: bucket maxima the shared layout is cut for
};
cudaError_t launch_fused(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* u_scratch,
                         cudaStream_t st);
size_t fused_smem_small(int dmax, int max_np);
size_t fused_smem_general(int max_np, int max_dpad, int threads, bool rot_in_smem);
int small_dmax_for(int dim);  // 0 when the small kernel does not apply
size_t fused_smem_tile(int max_np, int max_dpad, int threads, bool rot_smem);
// MLP objective (k_mlp.cu): its executors' rows (InstDesc.tc_row = first row)
struct MlpPlan {
    const int* execs;      // device [n_exec]
    int n_exec;
    const int* row_exec;   // device [n_rows] row -> executor
    int n_rows;
    int* topk_all;         // device [n_indiv] pbest pools
    float* uscr;           // trial rows (population layout)
    float* fu;             // trial fitness [n_indiv]
    const float* x;        // inputs [256][16]
    const float* y;        // targets of every MLP problem ([256][2] at InstDesc.aux)
    int max_dpad;
    int tc;                // evaluation: 0 FP32 CUDA cores (k_mlp_eval), 1 BF16 / 2 bf16x3 tensor cores (k_mlp_tc)
    int sms;               // CTAs of k_mlp_tc (one per SM)
};
// The GEMM pipeline's bounded mbarrier wait on its own (rounds 0: the
// pipeline's limit); out[0] completed, out[1] SM cycles; timeout latched in *status.
cudaError_t launch_wait_check(uint32_t rounds, int arrive, long long* out, int* status, cudaStream_t st);

cudaError_t launch_mlp_generation(const StepArgs& a, const MlpPlan& p, cudaStream_t st);
// f of the rows `rows` (population layout) of every MLP executor into f_out (fitness layout), in
// the plan's precision (a timeout of the tensor-core kernel is latched in *status)
cudaError_t launch_mlp_eval(const InstDesc* desc, const MlpPlan& p, const float* rows, float* f_out, int* status,
                            cudaStream_t st);
// the tensor-core evaluation alone (k_mlp_tc.cu)
cudaError_t launch_mlp_eval_tc(const InstDesc* desc, const MlpPlan& p, const float* rows, float* f_out, int* status,
                               cudaStream_t st);
cudaError_t launch_mlp_inputs(float* X, cudaStream_t st);
cudaError_t launch_mlp_targets(const float* X, const float* teacher, int h, float* Y, cudaStream_t st);
cudaError_t launch_fused_tile(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* u_scratch,
                              cudaStream_t st);

// Large-D executors on the tensor cores (tc_rotate.cu).
// Per-problem near-tie lists of the tensor-core path (device arrays of a
// TcPlan); tie_cnt null: one flat list instead.
struct TieLists {
    const int* prob_tp;   // problem -> index among the problems on the path
    const int* tp_row0;   // per such problem: start of its list
    int* tie_cnt;         // per such problem: ties listed
    long long* tie_off;   // population offset of each listed tie's row
};

struct TcPlan {
    const int* execs;        // device [n_exec] executors of the bucket
    int n_exec;
    const int* row_exec;     // device [n_rows] operand row -> executor (InstDesc.tc_row = first row)
    int n_rows;
    const int* tiles;        // device [n_tiles][2]: tensor cores (first operand row, rows <= 128) over the
                             // rows of one problem; FP32 GEMM (executor, first individual) of 64-row tiles
    int n_tiles;
    const long long* brow;   // device [n_prob] first B row of each problem
    int* topk_all;           // device [n_indiv] pbest pools
    float* uscr;             // trial rows (population layout)
    float* fu;               // trial fitness [n_indiv]
    void *aq, *aq_lo, *bq, *bq_lo;  // operands: BF16 (hi, lo) or e4m3 bytes
    float* ascale;           // FP8: per operand row, max|d| / 448
    float* bscale;           // FP8: per problem, max|R| / 448
    int fp8;                 // 1: e4m3 operands (kind::f8f6f4)
    int simt;                // 1: FP32 GEMM on the CUDA cores (k_rot_simt, 64-row tiles, no operands)
    int* tie_list;           // device [n_rows] rows whose selection is a near tie (fused path: fitness index)
    long long* tie_off;      // device [n_rows] fused path: population offset of each near tie's row
    int* tie_count;          // device counter
    int tie_ctas;            // CTAs of the tie kernel
    int kp, split, max_dpad;
    int fused;               // BF16 with FP32 ties, four kernels per generation: 1 k_tc_rank, k_tc_trial2,
                             // k_tc_sel, k_tc_ties2 (kp <= 256); 2 the same with k_rot_tc selecting (kp > 256)
    int* next_tile;          // device counter of k_tc_sel's tile queue
    int n_tp;                // problems with executors on this path
    const int* prob_tp;      // device [n_prob]: index among them (-1: none)
    const int* tp_row0;      // device [n_tp]: first operand row of each (start of its tie list)
    int* tie_cnt;            // device [n_tp]: near ties listed per problem
    int* chunk_ctr;          // device counter of k_tc_ties2's chunk queue
    int gen_ctas;            // CTAs of k_tc_sel (one per SM)
    unsigned long long* tie_total;  // device counter: near ties decided (read and cleared by the profile read)
    int* tie_done;           // device [n_rows] plan mode 2: row groups finished per tie chunk (kept at zero)
    float* tie_zs;           // device [n_rows][2][round_up(max_dpad, 4)] plan mode 2: z and dz of listed ties
    int wide_ctas;           // plan mode 2: CTAs of k_tc_ties_wide (as many as are resident at once)
    int4* trial_rec;         // device [n_rows][4] draw records (k_tc_rank -> k_tc_trial2; k_tc_sel in plan mode 1),
                             // written where k_tc_trial2 builds the rows: plan mode 1, narrow FP32 rows
    const int4* tmeta;       // device [n_tiles][2] tensor cores: (first row, rows, D, D_pad), (objective, problem)
    CUtensorMap mapA, mapB, mapAlo, mapBlo;
};
bool tc_make_map(CUtensorMap* map, const void* base, long long rows, int kp, int box_rows, int esz);
size_t tc_gemm_smem(bool split);
cudaError_t launch_tc_pack_rot(const float* rot, long long rot_off, int dim, int dpad, int kp, int np_rows, void* bq,
                               void* bq_lo, long long brow, int fp8, unsigned* amax, float* bscale, cudaStream_t st);
// Fitness of the population rows of every tensor-core executor, by the
// rotation GEMM in the plan's precision (written into fit).
cudaError_t launch_tc_eval(const InstDesc* desc, const TcPlan& p, const float* pop, const float* shift,
                           const float* rotT, float* fit, int* status, cudaStream_t st);
// FP32 rotation GEMM + objective on the CUDA cores (k_gemm32.cu): f of the
// rows `rows` (population layout) of every 64-row tile into f_out
// (columns of Z per chunk: the narrowest of 64, 128, 256 that covers max_dpad)
size_t rot_simt_smem(int max_dpad);
cudaError_t launch_rot_simt(const InstDesc* desc, const int* tiles, int n_tiles, const float* rows, const float* shift,
                            const float* rotT, float* f_out, int max_dpad, cudaStream_t st);
// The four-kernel generation (tc_fused.cu): whether the shared memory of
// k_tc_sel holds operands of kp BF16 elements, and one generation of every
// tensor-core executor -- k_tc_rank (pbest pools), k_tc_trial2 (trial and
// operand rows), k_tc_sel (GEMM, objective, selection, commit), k_tc_ties2
// (near ties) in plan mode 1; for operands wider than 256 (plan mode 2)
// k_tc_rank, k_tc_trial, k_rot_tc in selection mode and k_tc_ties_wide.
// ev (may be null): five events, before each launch and after the last.
bool tc_fused_fits(int kp);
// CTAs of k_tc_ties_wide resident on the device at once for vectors of max_dpad (0 on a CUDA error)
int tc_ties_wide_ctas(int max_dpad);
// k_tc_trial alone (trial rows and BF16 operand rows, a warp per row): the
// trial kernel of plan mode 2
cudaError_t launch_tc_trial_rows(const StepArgs& a, const TcPlan& p, cudaStream_t st);
// k_tc_trial2 alone (16 rows per CTA): trial rows, and BF16 operand rows of kp
// elements when aq is set; trec: the draw records k_tc_rank wrote (null: drawn here)
cudaError_t launch_tc_trial_rows32(const StepArgs& a, const TcPlan& p, void* aq, const int4* trec, cudaStream_t st);
// k_tc_rank alone: pbest pools, and the queues and per-problem tie counts of the generation zeroed;
// with trec, the rows' draw records as well
cudaError_t launch_tc_rank(const StepArgs& a, const TcPlan& p, int4* trec, cudaStream_t st);
// The near ties listed per problem, FP32 difference form: k_tc_ties2 when every
// D_pad <= 256, else k_tc_ties_wide (whose scratch the plan must hold)
cudaError_t launch_tc_ties_batched(const StepArgs& a, const TcPlan& p, cudaStream_t st);
// k_rot_tc with the selection in its epilogue (BF16): decisions against the stored
// fitness, clear acceptances committed, near ties listed per problem for k_tc_ties2
cudaError_t launch_rot_tc_select(const StepArgs& a, const TcPlan& p, cudaStream_t st);
cudaError_t launch_tc_fused_generation(const StepArgs& a, const TcPlan& p, cudaStream_t st,
                                       cudaEvent_t* ev = nullptr);
// ev (may be null): six events recorded before the prologue, trial, GEMM,
// selection and tie kernels and after the last.
cudaError_t launch_tc_generation(const StepArgs& a, const TcPlan& p, cudaStream_t st, cudaEvent_t* ev = nullptr);

// Evolver.
cudaError_t launch_outer_init(int n_groups, int n_out, Key key, float* opop, float* ofit, cudaStream_t st);
cudaError_t launch_outer_trial(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                               const float* opop, float* trial, float* theta, cudaStream_t st);
cudaError_t launch_outer_select(int n_groups, int n_out, float* opop, float* ofit, const float* trial,
                                const float* meta_fit, int tstride, cudaStream_t st);
cudaError_t launch_cso_move(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                            const float* opop, const float* ofit, float* trial, float* theta, cudaStream_t st);
cudaError_t launch_cso_select(int n_groups, int n_out, float* opop, float* ofit, const float* trial,
                              const float* meta_fit, cudaStream_t st);
cudaError_t launch_nes_sample(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen, float* trial,
                              float* theta, cudaStream_t st);
cudaError_t launch_nes_update(int n_groups, int n_out, float* opop, float* ofit, float* trial, const float* meta_fit,
                              cudaStream_t st);
cudaError_t launch_pso_move(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                            const float* opop, const float* ofit, float* trial, float* theta, cudaStream_t st);

}  // namespace metade
