// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "../../include/fmmcph.h"

namespace fmmcph {

// Every device allocation of the library goes through here, so that a test can make one fail
// (fmm_inject_alloc_failure) and check the FMM_ERR_OOM paths.
cudaError_t device_alloc(void** p, size_t bytes);

// NVTX range "fmm:<stage>" around the host-side launches of one stage of an evaluation, so that
// a profiler attributes the kernels to stages (ncu --nvtx --nvtx-include "fmm:near/").  Without
// an attached tool the calls do nothing.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// The bounds-checked build's per-file words (bounds.cuh): the source line of the first failed
// index check since the last call, 0 for none (always 0 in the normal build).
int bc_take_kernels();
int bc_take_m2l();
int bc_take_translate();

constexpr int kMaxP = FMM_MAX_P;
constexpr int kMaxDepth = 7;
constexpr int kLeafMomStride = 8;  // floats per leaf in Handle::leafmom
constexpr int kRootDoubles = 8 + 5 * 64 + 4 + 40;  // Handle::root beyond nc: Q D T, k_qdt partials, FP32 copies, k_final totals + ticket
constexpr int kNumOps = 343;  // M2L offsets o in {-3..3}^3 (the inner 27 slots unused)
constexpr int kNumStages = 11;  // the stage intervals fmm_stage_times reports
constexpr int kNumEvents = 24;  // profiling: timing events recorded per evaluation

inline int ncoef(int p) { return (p + 1) * (p + 1); }
inline int ncoef_padded(int p) { return (ncoef(p) + 15) / 16 * 16; }
inline int op_index(int ox, int oy, int oz) { return (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3); }

// A brick of target boxes of one level and octant class for the FP32 CUDA-core M2L: the boxes
// (i0 + i, j0 + j, k0 + k), 0 <= i < bx, j < by, k < bz, of the class sub-grid (n = 2^(level-1)
// boxes per axis).
struct F32Brick {
    int level, cls, i0, j0, k0, bx, by, bz;
};

struct M2LTile {
    int level;
    int cls;          // child octant class of the target boxes (0..7)
    int parent0;      // first parent index (Morton, at level-1)
    int nparents;     // parents in this tile
};

// A fixed translation operator packed for the tensor-core M2M / L2L (translate_tc.cu)
struct TranslateOp {
    uint8_t* dev = nullptr;
    size_t bytes = 0;
    int Mtot = 0, K = 0, nmt = 0, nkc = 0;
};

struct Handle {
    int device = 0;
    fmm_box box{};
    int periodic = 0, p = 0, depth = 0;
    int nc = 0, ncp = 0;
    int precision = FMM_FP32;
    bool hamiltonian = false;  // Hamiltonian interpolation within sites (intra-site correction)
    double ke = 138.935458;
    double s_bin = 0.0;  // 2^depth / L
    int lmin = 2;        // first level with M2L
    // operators (device)
    float* T = nullptr;        // [343][ncp(k)][ncp(j)]  M2L, transposed (input row k, output col j)
    float* A = nullptr;        // [8][ncp][ncp] M2M transposed
    float* B = nullptr;        // [8][ncp][ncp] L2L transposed
    float* B2 = nullptr;       // [ncp][8 ncp] L2L, all octants side by side
    double* Ad = nullptr;      // [8][nc][nc] M2M row-major, FP64 (root step)
    double* Lam = nullptr;     // [nc][nc] lattice, FP64 row-major
    TranslateOp m2m_tc, l2l_tc;  // mixed precisions: M2M and L2L on the tensor cores
    M2LTile* tiles = nullptr;  // M2L work list
    int ntiles = 0;
    // FP32 CUDA-core M2L (ncp <= 128): bricks of target boxes of one level and octant class
    F32Brick* bricks = nullptr;
    int nbricks = 0;
    float* m2l_part = nullptr;  // [8][nbox_total][ncp] partials per source class
    // tree storage
    std::vector<long> lvl_off;  // box offset of each level
    long nbox_total = 0;
    float* M = nullptr;  // [nbox_total][ncp]
    float* L = nullptr;
    // atoms
    int cap = 0, n = 0, K = 0;
    float *qA = nullptr, *qB = nullptr, *lam = nullptr;
    float *qC = nullptr, *qD = nullptr;  // four-form sites (Eq. 2): forms C and D
    int nforms = 2;                      // charge forms per site: 2 (Eq. 1) or 4 (Eq. 2)
    int ncoord = 1;                      // lambda coordinates per site: 1 or 2 (lambda_p, lambda_t)
    float* dqt = nullptr;                // four-form sites: dq/dlambda_t per sorted atom (dq holds dq/dlambda_p)
    const float* lam_bound = nullptr;
    int32_t* site = nullptr;
    int* site_ptr = nullptr;    // [K+1]
    int* site_atoms = nullptr;  // [#site atoms], input indices grouped by site, ascending
    int site_cap = 0, lam_cap = 0;
    uint32_t *key = nullptr, *kA = nullptr, *kB = nullptr, *vA = nullptr, *vB = nullptr;
    uint32_t *perm = nullptr, *inv = nullptr, *sorted_key = nullptr;
    uint32_t *start = nullptr, *count = nullptr;
    uint32_t* leafcnt = nullptr;  // [leafcnt_words(nleaf)] per-leaf, then per-tile counters of the binning step, zero between calls
    float4* pos = nullptr;
    float* dq = nullptr;
    float* phis = nullptr;   // sorted-order potential (without k_e)
    float4* near = nullptr;  // sorted-order near-field potential and gradient (k_p2p -> k_far_out)
    // the near field's work items (leaf, tile) of leaves above 64 atoms: count in [0].x, then the
    // items (listed by the binning)
    int2* near_items = nullptr;
    int near_items_cap = 0;
    float2* epart = nullptr;  // per-block (hi, lo) partial sums of q phi
    int epart_cap = 0;
    float* leafmom = nullptr;   // [nleaf][kLeafMomStride] periodic: leaf moments for the Q, D, T sums
    double* root = nullptr;     // [nc] FP64 root multipole, then [5] Q D T at root+nc
    // Hamiltonian interpolation: h of the periodic pair potential (normalised root local
    // expansion, [ncp]), per-site energy and dV/dlambda corrections ([K][2]), and per-atom
    // per-form terms of the Hamiltonian correction's charge gradient (input order) for the adjoint
    float* hi_coef = nullptr;
    double* hi_site = nullptr;  // [K][3]: energy, dV/dlambda_p (or dV/dlambda), dV/dlambda_t corrections
    float4* hi_g = nullptr;  // per atom (input order), per form X: sum_j (q^X_j - q_j) psi_ij
    int hi_cap = 0, hi_kcap = 0;
    int* status = nullptr;
    float* work = nullptr;  // split-K partial products (8 x the largest M2M output level)
    bool charges_set = false;
    // limit (clock cycles) of the pipeline waits of the tensor-core M2L, M2M and L2L and of the
    // near field's staging waits; 0 = the default (about 2 s), a small value lets a test make
    // the waits expire (fmm_set_wait_limit)
    long long wait_limit = 0;
    // test hook (fmm_inject_copy_loss): FMM_LOSE_* bits of the kernels whose bulk copies are
    // announced on their barriers but not issued, so that their bounded waits run out
    int copy_loss = 0;
    // kernel tiles (fmm_options): the tensor-core M2L's rows per CTA (0 = 192) and the near
    // field's leaves (warps) per block (2, 4 or 8)
    int m2l_rows = 0;
    int p2p_warps = 4;
    // profiling
    int profiling = 0;  // 0 off, 1 per-stage events, 2 the same with every stage serialised
    cudaEvent_t ev[kNumEvents]{};  // a pool of timing events, taken in launch order
    int ev_used = 0;
    int stage_ev[kNumStages][2]{};  // per stage: the pool events that bracket it, -1 if not run
    bool ev_valid = false;
    // the multipole chain runs on `chain` (highest priority) while the near field runs on the
    // caller's stream; fork/join by events.  With the tensor-core M2L and coarse levels below
    // the two finest, `side` (also highest priority) takes the coarse levels' M2L, the periodic
    // root and the coarse levels' L2L, concurrently with the finest levels' M2L on `chain`.
    cudaStream_t chain = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t m2m_ev = nullptr, side_ev = nullptr;
    // one evaluation as a CUDA graph (fmm_eval, fmm_eval_host): captured on `gcap` the second time
    // in a row the same buffers come, replayed on the caller's stream while they and the handle's
    // launch state (generation `gen`, bumped by every call that changes it) stay the same
    cudaStream_t gcap = nullptr;
    struct EvalGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key[5]{};
        unsigned long long gen = 0, used = 0;
    };
    EvalGraph g_slot[2];           // the graphs of the two most recent buffer sets
    const void* g_hist[2][5]{};    // the buffer sets of the last two eager evaluations
    unsigned long long g_hist_gen[2] = {~0ull, ~0ull};
    int g_hist_next = 0;
    unsigned long long gen = 0, g_tick = 0;
    bool g_off = false;  // a capture failed once: evaluations stay eager launches
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // the end of the last evaluation's kernels and its stream: an evaluation on another stream
    // waits for it (the handle's buffers are shared), not for what that stream does afterwards
    cudaEvent_t eval_ev = nullptr;
    cudaStream_t eval_last = nullptr;
    bool eval_ev_valid = false;
    // host staging for fmm_eval_host(_async): two device sets used in turn, so that the copy
    // of one call's positions (on h2d) overlaps the previous call's evaluation
    float* hx_dev[2] = {nullptr, nullptr};
    float* hF_dev[2] = {nullptr, nullptr};
    float* hdV_dev[2] = {nullptr, nullptr};
    double* hE_dev[2] = {nullptr, nullptr};
    int hdV_cap = 0;
    int host_cap = 0;
    int h_next = 0;
    cudaStream_t h2d = nullptr;
    cudaEvent_t hx_ev[2] = {nullptr, nullptr}, hfree_ev[2] = {nullptr, nullptr};
    void* tc = nullptr;  // tensor-core M2L state (m2l_tc.cu)
};

// kernels.cu
void upload_constants(int p);
void near_configure(Handle* h);  // the near field's shared-memory limit and grid (per handle)
int launch_eval(Handle* h, const float* x, double* E, float* F, float* dVdl, float* phi,
                cudaStream_t st);
int leafcnt_words(int nleaf);  // the binning's counters: one per leaf, one per scan tile
int launches_per_eval(const Handle* h);
void f32_bricks(int lmin, int depth, std::vector<F32Brick>& out);  // the FP32 M2L's work list
void launch_adjoint(Handle* h, const double* gbar, const float* F, const float* phi,
                    const float* dVdl, float* gx, float* const* gq /*[4] forms, may be null*/, float* glam,
                    cudaStream_t st);
// translate_tc.cu
TranslateOp translate_pack(const std::vector<float>& W, int Mtot, int K);  // W row-major [Mtot][K]
void translate_free(TranslateOp& op);
void translate_configure();
void translate_tc(const TranslateOp& op, const float* X, int ldx, int N, float* C, int ldc, bool accumulate,
                  int* status, cudaStream_t st, int ksplit = 1, float* work = nullptr, long long wait_limit = 0,
                  bool lose_copies = false);
// m2l_tc.cu
bool m2l_tc_supported(const Handle* h);
bool m2l_tile_rows_ok(int rows);  // 0 (the default) or a width the kernel is instantiated for
int m2l_tc_setup(Handle* h, const std::vector<float>& T_rowmajor);  // [343][nc][nc], output-major
void m2l_tc_free(Handle* h);
int m2l_tc_launches(const Handle* h);
// the M2L of tree levels lo .. hi (clamped to the handle's levels): the pack of their
// multipoles (kM2lPack), then the MMA kernel over their tiles (kM2lMma)
constexpr int kM2lPack = 1, kM2lMma = 2;
void launch_m2l_tc(Handle* h, cudaStream_t st, int lo, int hi, int parts = kM2lPack | kM2lMma);

}  // namespace fmmcph
