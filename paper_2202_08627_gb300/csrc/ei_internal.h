// Internal declarations shared by the CUDA translation units of libei.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "../../include/ei.h"

namespace ei {

// Debug build (-DEI_DEVICE_CHECKS, built beside the library as
// libei_check.so): the kernels whose loads rely on zero margins sized on the
// host (projector, adjoint) check every data-dependent index; a failed check
// records EI_ERR_DEVICE_CHECK in the device status word and the access is
// clamped into its array, so it never leaves it.  In the regular build the
// checks compile away.
#ifdef EI_DEVICE_CHECKS
constexpr bool kDeviceChecks = true;
#else
constexpr bool kDeviceChecks = false;
#endif

#ifdef __CUDACC__
// i when lo <= i <= hi; otherwise (check builds only) the status word records
// the failure and the nearest bound is returned.
__device__ __forceinline__ int checked_index(int i, int lo, int hi, int *status)
{
    if (kDeviceChecks && (i < lo || i > hi)) {
        if (status) atomicCAS(status, 0, (int)EI_ERR_DEVICE_CHECK);
        return i < lo ? lo : hi;
    }
    return i;
}
#endif

// An NVTX range for the lifetime of the object (phases of the library's
// calls, visible to profilers that record NVTX, e.g. ncu --nvtx).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-slice constants, resident in device memory (one entry per slice).
struct SliceInfo {
    int n, n_theta, n_det, n_dp;
    float pitch, inv_pitch;  // voxel = detector pitch (cm) and its inverse
    int ang_off;             // first angle of the slice in the angle tables
    int pix_off;             // first pixel of the slice in the pixel table (n_dp stride)
    int marg;                // zero entries on each side of a packed gradient-sinogram row
    int gw;                  // packed gradient-sinogram row width: n_dp + 2 marg entries
    int det_off;             // first pixel of the slice in per-pixel user arrays (n_det stride)
    int64_t vol_off;         // float4 elements (vol layout)
    int64_t pp_off;          // entries of the packed volume copies: n rows of n + 1
    int64_t gp_off;          // entries of the packed gradient sinogram: n_theta rows of gw
    int64_t sino_off;        // pixels: base of [n_theta][n_dp] (user sino4 and every plane)
    int64_t proj_off;        // floats: 3 planes
    int64_t meas_off;        // floats: n_m planes
};

// Pair-packed arrays.  Sampling a linear interpolation needs two neighbouring
// (mu, delta, sigma) triples; entry e of a packed row holds the triple at
// e - 1 and the one at e as a float4 (mu0, delta0, sigma0, mu1) plus a float2
// (delta1, sigma1), so one sample is 24 bytes in two loads.
//   packed volume copy (projector input): row o, entry e = i + 1 holds voxel
//     i of that row and the difference voxel(i + 1) - voxel(i), as
//     (mu0, delta0, sigma0, mu1 - mu0) + (delta1 - delta0, sigma1 - sigma0),
//     i in [-1, n - 1] (voxels outside the slice are zero), so a sample is
//     one FMA per channel; xpA/xpB row-major (o = r, i = c), xtA/xtB
//     transposed (o = c, i = r).
//   packed gradient sinogram (adjoint input): row a, entry e holds pixels
//     j = e - marg and j + 1; pixels outside [0, n_det) are zero, and the
//     margin covers every pixel a voxel of the slice can project to.

// Per (slice, angle) constants, computed on the host in FP64.
// The ray of pixel j samples the "outer" voxel index o = 0..n-1 (rows when
// |cos| >= |sin|, else columns) at inner position s(o) = (j - hd) * inv_dom +
// k0 + o * p1 (inner index units: columns, resp. rows).
struct AngleInfo {
    double inv_dom;     // 1/cos (row-dominant) or -1/sin (column-dominant)
    double k0;          // hn - hn * p1
    double p1;          // tan (row-dominant) or cot (column-dominant)
    double inv_p1;      // 1/p1, 0 when p1 == 0
    long long p1_fx;    // round(p1 * 2^32)
    long long cos_fx;   // round(cos * 2^32)
    long long sin_fx;   // round(sin * 2^32)
    float cosf, sinf;   // cos, sin
    float inv_ch, pch;  // 1/ch and pitch/ch, ch = max(|cos|, |sin|)
    int col_dom;        // 1 when |sin| > |cos|
    int pad_;
};

// The constants of angle th for a slice of n x n voxels of the given pitch
// (the setup on the host and the allocation-free path's table kernel share it).
__host__ __device__ inline AngleInfo make_angle_info(double th, int n, double pitch)
{
    const double TWO32 = 4294967296.0;
    const double hn = 0.5 * (n - 1);
    const double ct = cos(th), st = sin(th);
    const double ch = fmax(fabs(ct), fabs(st));
    AngleInfo an{};
    an.col_dom = fabs(st) > fabs(ct) ? 1 : 0;
    if (!an.col_dom) {
        an.inv_dom = 1.0 / ct;
        an.p1 = st / ct;
    } else {
        an.inv_dom = -1.0 / st;
        an.p1 = ct / st;
    }
    an.k0 = hn - hn * an.p1;
    an.inv_p1 = an.p1 != 0.0 ? 1.0 / an.p1 : 0.0;
    an.p1_fx = llrint(an.p1 * TWO32);
    if (an.p1_fx == 0) an.p1 = 0.0, an.inv_p1 = 0.0;
    an.cos_fx = llrint(ct * TWO32);
    an.sin_fx = llrint(st * TWO32);
    an.cosf = (float)ct;
    an.sinf = (float)st;
    an.inv_ch = (float)(1.0 / ch);
    an.pch = (float)(pitch / ch);
    return an;
}

struct ModelConsts {
    float z_over_p;       // shift in periods per unit dR[delta]/dt
    float kappa;          // IC variance per unit R[sigma]
    int n_m;
    float m[EI_MAX_NM];
};

// Work decomposition sizes.
constexpr int ADJ_TC = 32;                 // adjoint tile: 32 columns x (8 x passes) rows
constexpr int ADJ_MAX_TR = 128;            // tallest adjoint tile among the variants
constexpr int ADJ_THREADS = 256;
constexpr int PREP_TILE = 32;              // staging tile
constexpr int EI_MAX_LBFGS_M = 32;         // largest L-BFGS memory (ei_solve_opts.lbfgs_m)
constexpr int VEC_BLK = 4096;              // float4 per vector-op block (one slice per block)
constexpr int VEC_THREADS = 256;

// Kernel variants the autotuner chooses among (instantiated in k_project.cu /
// k_backproject.cu).  Each has its own work decomposition.
constexpr int N_FWD_VARIANTS = 14;          // projector tile (rays x angles, warp shape, unroll, staging)
constexpr int N_ADJ_VARIANTS = 14;         // adjoint voxels per thread and occupancy
// Adjoint variants that read the mirror-interleaved gradient layout.
inline bool adj_mirror_layout(int id) { return id >= 11; }
void project_variant_shape(int id, int *rays, int *angles);
int backproject_variant_rows(int id);
int backproject_variant_items(int id, int n);

struct FwdVariant {
    int id = 0;
    const int *prefix = nullptr;   // device [n_slices + 1] work-item prefix sums
    int total = 0;
};
struct AdjVariant {
    int id = 0;
    const int *prefix = nullptr;
    int total = 0;
};

// Device-side view of a geometry, passed to kernels by value.
struct DevGeom {
    const SliceInfo *slices;
    const AngleInfo *ang;        // [sum n_theta]
    const float *m_o;            // [sum n_theta]
    const float4 *pix;           // [sum n_dp]: (A, c, w, m_r)
    const int *ic_prefix;        // [n_slices + 1] work-item prefix sums (IC rows,
    const int *prep_prefix;      // staging tiles, vector blocks; the projector's and
    const int *vec_prefix;       // adjoint's belong to their variants)
    int n_slices;
    int total_ic, total_prep, total_vec;
    int max_ndp, max_n_theta;
    ModelConsts mc;
    // solver view with Eq. 4's offsets among the unknowns (null otherwise): per
    // slice vec_nvb[s] volume blocks then the blocks of an offsets segment of
    // off_len[s] float4 starting at element off_start[s] of the solver vectors
    const int *vec_nvb = nullptr;
    const int64_t *off_start = nullptr;
    const int *off_len = nullptr;
    // sampled flat IC (null: the Gaussian of pix): [sum n_det][flat_k] samples
    // f(t, k / flat_k) over one mask period, rows in the order of det_off
    const float *flat_tab = nullptr;
    int flat_k = 0;
    // device status word of the kernels' bounded waits and (check builds)
    // bounds checks; may be null
    int *status = nullptr;
    // layout of the packed gradient sinogram the IC kernels and k_pack_sino
    // write: 0 pair-packed (entry j: pixels j and j + 1), 1 mirror-interleaved
    // (entry j: pixels j and n_det - 1 - j), as the selected adjoint variant reads
    int gmirror = 0;
};

// Launch modes of the projector and the adjoint: one block per work item; a
// persistent GPU-sized grid whose blocks take items from one counter; or a
// persistent grid whose blocks first take the items of their own SM's
// contiguous chunk of the work list (so the blocks resident on one SM work on
// neighbouring items and share L1 lines), then those of the other chunks.
enum LaunchMode { LAUNCH_PER_ITEM = 0, LAUNCH_PERSISTENT = 1, LAUNCH_SM_CHUNKS = 2 };
constexpr int N_LAUNCH_MODES = 3;
constexpr int MAX_SM_CHUNKS = 1024;        // per-SM chunk counters (>= %nsmid)

#ifdef __CUDACC__
// Next work item of an SM-chunked launch for the block's thread 0: the list
// [0, total) is cut into nchunk contiguous chunks; the block takes the next
// item of chunk (sm + k) % nchunk, k = *k_state (0: its own SM's chunk) and
// advances k when that chunk is exhausted; -1 when every chunk is.  Each call
// makes at most nchunk atomic increments; nothing waits.
__device__ __forceinline__ int sm_chunk_next(int total, int *counters, int sm, int nchunk,
                                             int *k_state)
{
    while (*k_state < nchunk) {
        const int c = (sm + *k_state) % nchunk;
        const int lo = (int)((long long)total * c / nchunk);
        const int hi = (int)((long long)total * (c + 1) / nchunk);
        if (lo < hi) {
            const int idx = atomicAdd(counters + c, 1);
            if (lo + idx < hi) return lo + idx;
        }
        ++*k_state;
    }
    return -1;
}

// The SM a block runs on, and the number of SM ids (PTX special registers).
__device__ __forceinline__ int sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int sm_id_count()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(r));
    return (int)r < MAX_SM_CHUNKS ? (int)r : MAX_SM_CHUNKS;
}

// Slice owning work item `item`: the largest s with prefix[s] <= item.
__device__ __forceinline__ int find_slice(const int *prefix, int n_slices, int item)
{
    int lo = 0, hi = n_slices - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}
#endif

struct Solver;

}  // namespace ei

// The opaque handle.
struct ei_geometry {
    int n_slices = 0;
    int n_m = 0;
    int device = 0;
    std::vector<ei::SliceInfo> h_slices;
    std::vector<int> h_vec_prefix;
    float lambda[3], scale[3];
    ei::DevGeom dg{};
    std::vector<void *> allocs;    // device allocations owned by the geometry
    // workspace for objective / forward evaluations
    float4 *xpA = nullptr, *xtA = nullptr;   // packed volume copies (times mult)
    float2 *xpB = nullptr, *xtB = nullptr;
    float *proj = nullptr;         // proj layout
    float4 *gA = nullptr;          // packed gradient sinogram
    float2 *gB = nullptr;
    double *part_ic = nullptr;     // [total_ic]
    double *part_reg = nullptr;    // [total_vec] regulariser partial sums
    double *S_dev = nullptr;       // [n_slices]
    int64_t vol_count = 0, pp_count = 0, gp_count = 0, proj_count = 0, sino4_count = 0,
            meas_count = 0;
    int64_t workspace_bytes = 0;
    ei::Solver *solver = nullptr;      // allocated on first ei_reconstruct
    // kernel variants (autotuner) and persistent launches
    ei::FwdVariant fwd_variant;
    ei::AdjVariant adj_variant;
    const int *fwd_prefixes[ei::N_FWD_VARIANTS] = {};
    int fwd_totals[ei::N_FWD_VARIANTS] = {};
    const int *adj_prefixes[ei::N_ADJ_VARIANTS] = {};
    int adj_totals[ei::N_ADJ_VARIANTS] = {};
    int persistent = 0;                // launch mode (LaunchMode) of projector and adjoint
    int *sm_counters = nullptr;        // [MAX_SM_CHUNKS] chunk counters of LAUNCH_SM_CHUNKS
    int ic_variant = 0;                // 0: one block per row; 1: persistent, bulk-copy pipeline
    float link_gamma = 0.f;            // > 0: linked unknown h (mu = h, delta = gamma h, sigma = 0)
    int off_which = 0;                 // Eq. 4 offsets among the solver's unknowns (EI_OFFSET_*)
    float off_scale = 1.f;             // their solver scaling u = m / off_scale
    int ring_modes = 0;                // m_r steps orthogonal to the K lowest DCT-II modes
    float *shift_scratch = nullptr;    // [sino4_count] dS/dshift (ei_offset_grad, allocated on use)
    double *row_sums = nullptr;        // [total_ic]
    float *eq3_ker = nullptr;          // [sum n_det] Eq. 3 convolution kernels (allocated on use)
    float *flat_buf = nullptr;         // storage of dg.flat_tab (allocated on use)
    int64_t flat_cap = 0;              // its capacity in floats
    int *dev_status = nullptr;         // [1] device-side error status (bounded waits)
    int num_sms = 0;
    int *work_counter = nullptr;       // [2] work counters of the persistent kernels
    // work per slice, for the autotuner's cache key
    uint64_t shape_hash = 0;
    // tracing (ei_profile_enable): launch counter and event pairs per traced kernel
    bool prof_on = false;
    int64_t launches = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pairs[3];
};

namespace ei {

enum IcMode { IC_MODEL = 0, IC_OBJECTIVE = 1, IC_OBJECTIVE_GRAD = 2 };

enum TracedKernel { TK_PROJECT = 0, TK_IC = 1, TK_BACKPROJECT = 2 };

// Tracing helpers: count `n` launches; bracket a traced launch with events.
inline void count_launches(ei_geometry *g, int n) { g->launches += n; }
cudaEvent_t trace_begin(ei_geometry *g, cudaStream_t st);
void trace_end(ei_geometry *g, TracedKernel k, cudaEvent_t begin, cudaStream_t st);

// Kernel launchers (each returns cudaGetLastError()).
// Packed volume copies of mult * vol (row-major and transposed) in the workspace;
// linked: single-channel copies of mult.x * vol.x (the B arrays only).
cudaError_t launch_prep(const ei_geometry *g, const float4 *vol, float4 mult, bool linked,
                        const int *active, cudaStream_t st);
// proj = R[x] from the packed copies; link > 0 (after a linked prep): the three
// planes are (R[h], link R[h], 0).
cudaError_t launch_project(const ei_geometry *g, float *proj, float link, const int *active,
                           cudaStream_t st);
// IC model; in IC_OBJECTIVE_GRAD mode it writes the packed gradient sinogram, or
// with link > 0 only the single pair-packed sinogram g_mu + link g_delta (in gB).
cudaError_t launch_ic(const ei_geometry *g, const float *proj, const float *meas, float *s_mod,
                      double *part, IcMode mode, float link, const int *active, cudaStream_t st);
// Whether the bulk-copy IC variant's two row buffers fit in shared memory.
bool ic_pipe_fits(int max_ndp, int n_m);
// Single-shot retrieval + ramp filter into the packed gradient sinogram
// (the adjoint then gives the filtered back-projection).
cudaError_t launch_single_shot(const ei_geometry *g, const float *meas, cudaStream_t st);
cudaError_t single_shot_set_smem_limit();
// The paper's single-shot retrieval (Eq. 3) of the linked unknown from mask
// position m_index into the packed gradient sinogram (channels R[h], gamma R[h],
// 0, ramp-filtered with the FBP scale); ker: [sum n_det] scratch for the
// per-slice convolution kernels.
cudaError_t launch_single_shot_eq3(const ei_geometry *g, const float *meas, int m_index,
                                   float gamma, float *ker, cudaStream_t st);
bool single_shot_eq3_fits(const ei_geometry *g);
// Packed gradient sinogram from a user sino4 array.
cudaError_t launch_pack_sino(const ei_geometry *g, const float4 *sino4, cudaStream_t st);
// out = out_mult * R^T g + reg2 * v (g: the packed gradient sinogram; v may be null).
// link > 0 (the linked unknown h of Eq. 4; gB then holds the single sinogram
// g_mu + link g_delta that launch_ic wrote): out = (out_mult.x R^T g + reg2.x v.x,
// 0, 0, 0).
cudaError_t launch_backproject(const ei_geometry *g, const float4 *v, float4 *out,
                               float4 out_mult, float4 reg2, float link, const int *active,
                               cudaStream_t st);
// The regulariser's value: per vector block of dg (volume blocks; an offsets
// block of a solver view writes 0) the FP64 sum of sum_c reg1_c v_c^2 over its
// voxels, into part[block].
cudaError_t launch_reg_partials(const DevGeom &dg, const float4 *v, float4 reg1, double *part,
                                const int *active, cudaStream_t st);
// dS/dshift per sinogram pixel into shift (sino layout, one float per pixel) and its
// FP64 sum over each row into row_sum; then per slice dS/dm_o (the row sums) into
// g_mo [sum n_theta] and dS/dm_r (FP64 sums over angles) into g_mr [sum n_det].
cudaError_t launch_offset_grads(const ei_geometry *g, const float *proj, const float *meas,
                                float *shift, double *row_sum, float *g_mo, float *g_mr,
                                cudaStream_t st);
// First half of the above for the slices with active[s] (all when null):
// dS/dshift into shift, its row sums into row_sum.
cudaError_t launch_shift_grad(const ei_geometry *g, const float *proj, const float *meas,
                              float *shift, double *row_sum, const int *active, cudaStream_t st);
// S[s] = sum of part_ic over the slice's rows + sum of part_reg over its vector
// blocks reg_prefix[s] .. reg_prefix[s + 1] - 1 (device prefix table).
cudaError_t launch_finalize_objective(const ei_geometry *g, const double *part_ic,
                                      const int *reg_prefix, const double *part_reg, double *S,
                                      const int *active, cudaStream_t st);

// The constants an evaluation stages and finishes with.  scaled == false: the
// unknown is the physical x (regulariser lambda ||x / scale||^2); scaled ==
// true: u = x / scale (the solver's).  Linked mode: h in the mu lane.
struct EvalConsts {
    float4 mult;       // staging multipliers (projections of mult * v)
    float4 out_mult;   // adjoint: out = out_mult R^T g + reg2 v
    float4 reg2;
    float4 reg1;       // regulariser's value: sum_c reg1_c v_c^2
    float link;        // gamma of the linked unknown, 0 otherwise
};
EvalConsts eval_consts(const ei_geometry *g, bool scaled);

// S (and grad when non-null) for every active slice, on the geometry's workspace.
// scaled == false: v is the physical x (P = R x, grad wrt x, regulariser on x/scale).
// scaled == true:  v is u = x/scale (P = R (scale u), grad wrt u, regulariser on u).
cudaError_t evaluate(ei_geometry *g, const float4 *v, const float *meas, double *S_dev,
                     float4 *grad, bool scaled, const int *active, cudaStream_t st);

int reconstruct(ei_geometry *g, const float *s_exp, float *vol_inout, const ei_solve_opts *opts,
                ei_solve_report *report, cudaStream_t st);
// Remember the last CUDA error of this thread (reported by ei_last_error).
void record_error(cudaError_t e);
// Remember a formatted message as the last error of this thread.
void record_message(const char *fmt, ...);
// Select kernel variants (ids in range) and the launch mode.
void select_variants(ei_geometry *g, int fwd_id, int adj_id, int launch_mode);
void destroy_solver(ei_geometry *g);
// Checkpoint of the solver state (ei_solver_state_size / _save / _load).
size_t solver_state_size(const ei_geometry *g, int m);
int solver_save(const ei_geometry *g, void *buf, size_t bytes);
int solver_load(ei_geometry *g, int m, const void *buf, size_t bytes);

}  // namespace ei

#define EI_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return _e;                  \
    } while (0)
