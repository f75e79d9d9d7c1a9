/*
 * dpgb.h -- C ABI of the GB300 (sm_103a) Deep Potential engine.
 *
 * The library evaluates the energy E, forces F and virial Xi of a smooth-edition
 * Deep Potential (DeePMD-kit v2, arXiv 2304.09409):
 *
 *   neighbour list n(i) with a fixed per-type sel       (Sec. II.A.1 "Handling the
 *                                                        systems composed of multiple
 *                                                        chemical species"; Sec. III.B.1)
 *   environment matrix R with the switch s(r)           (Eqs. (rij), (switch))
 *   embedding G = N_{e,2}^{a_i,a_j}(s)  or its quintic  (Eqs. (G2), (NN), (compress))
 *   descriptor D = (1/Nc^2) G^T R R^T G_<               (Sec. II.A.1, se_e2_a; also se_e2_r,
 *                                                        se_e3 and the hybrids of se_e2_a with
 *                                                        either, see dp_model_config)
 *   E_i = F_0^{a_i}(D^i),  E = sum_i E_i                (Eq. (fitting_energy))
 *   F = -dE/dr,  Xi_ab = -sum_g dE/dh_ga h_gb            (Sec. II.A.2)
 *
 * and, for training and active learning, the parameter gradient of the loss of Eq. (loss)
 * (dp_param_grad, Sec. II.B) and the model deviation of an ensemble (dp_model_deviation,
 * Sec. II.C).
 *
 * Conventions shared by every entry point
 *   - Every call returns a status code (DP_OK = 0); nothing aborts.  On error,
 *     dp_last_error() gives a message for the calling thread.
 *   - Non-finite coordinates (NaN, Inf) are rejected with DP_E_ARG: host arrays before any
 *     work is launched, device arrays by a flag the list build raises (the frame's atoms are
 *     then binned as if at the origin, so no kernel leaves its buffers, and the call's results
 *     are not valid).
 *   - The caller owns every input and output buffer.  The library owns models,
 *     neighbour lists and the scratch memory it allocates for them.
 *   - Array arguments may be host or device pointers (detected per pointer).  Host
 *     inputs are copied to the device inside the call and host outputs are copied back
 *     before the call returns.  `box` is always a host pointer: it fixes the cell grid.
 *   - Coordinates are FP64 [natoms][3] (Angstrom), types are int32 [natoms] in
 *     [0, ntypes).  box is FP64 [3][3] row-major, row g is the cell vector h_g; box ==
 *     NULL means open boundaries (no periodic images).
 *   - Output atom order equals input atom order.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that return
 *     results synchronise that stream before returning.
 */
#ifndef DPGB_H
#define DPGB_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DP_OK 0
#define DP_E_ARG 1          /* invalid argument (null pointer, bad size, bad type, bad box)   */
#define DP_E_CUDA 2         /* a CUDA runtime call failed                                    */
#define DP_E_OOM 3          /* device memory could not be allocated                          */
#define DP_E_SEL_OVERFLOW 4 /* some atom had more neighbours of a type than sel: the list
                               keeps the sel nearest and the results are computed (warning) */
#define DP_E_TIMEOUT 5      /* a bounded device wait gave up                                 */
#define DP_E_RANGE 6        /* compressed model: some s fell outside the table (the last
                               piece was extrapolated; results are computed, warning)       */
#define DP_E_CAPACITY 7     /* more than DP_MAX_CANDIDATES atoms inside r_c of one atom     */
#define DP_E_UNSUPPORTED 8  /* configuration outside what the kernels implement              */

/* ---- precision of the network arithmetic ---- */
#define DP_PREC_FP64 0 /* every step in FP64                                                 */
#define DP_PREC_FP32 1 /* networks and contractions in FP32; FP64 for the pair distance, the
                          switch near r_c, the energy sum and the force/virial accumulation */
#define DP_PREC_TF32 2 /* as FP32, with the embedding and fitting GEMMs on TF32 tensor cores (FP32
                          accumulation); uncompressed models only                             */
#define DP_PREC_BF16 3 /* as FP32, with the network GEMMs on BF16 tensor cores (FP32 accumulation):
                          uncompressed, the embedding and fitting layers; compressed, the fitting
                          net and the interval-moment contraction (FP16 operands)              */

#define DP_MAX_TYPES 8
#define DP_MAX_LAYERS 8
#define DP_MAX_CANDIDATES 1024 /* atoms within r_c of one atom the list builder can hold */

/* Descriptors (Sec. II.A.1) */
#define DP_DESC_SE_E2_A 0   /* D = T T_<^T, T = G^T R / Nc, R rows (s, s x/r, s y/r, s z/r): M x M_< */
#define DP_DESC_SE_E2_R 1   /* R reduced to its radial column s: D = G^T s / Nc, M values          */
#define DP_DESC_HYBRID_R 2  /* se_e2_a part, then an se_e2_r part: D = [D_a, D_r]                  */
#define DP_DESC_SE_E3 3     /* D = (R R^T) : G / Nc^2, G_jk = N^{a_j,a_k}(R_j . R_k): M values      */
#define DP_DESC_HYBRID_E3 4 /* se_e2_a part, then an se_e3 part: D = [D_a, D_e3]                   */

/* Model hyper-parameters (Sec. II.A.1, II.A.2, II.A.6).  embed[] are the embedding-net
 * widths (input width 1 is implied), fit[] the fitting-net hidden widths (a final linear
 * width-1 layer is implied).  ResNet skips follow Eq. (NN) with w_hat = 1.
 * rcut, rcut_smth, sel, embed describe the descriptor's (first) part; axis is read by
 * se_e2_a parts only.  Hybrids take their second part from rcut_2, rcut_smth_2, sel_2,
 * n_embed_2, embed_2.  Every part reads one neighbour list built with the larger cutoff and,
 * per type, the larger sel of the parts: a part's own list (its sel[t] nearest type-t
 * neighbours within its cutoff) is the prefix of each type block closer than its cutoff.
 * se_e3 nets are indexed by the two neighbours' types (ntypes^2 nets, type_one_side not
 * applicable).  The fitting-net input is the concatenation of the parts' D.  Descriptors other
 * than se_e2_a run on the CUDA-core path only (DP_PREC_FP64 / DP_PREC_FP32, uncompressed);
 * other combinations are refused with DP_E_UNSUPPORTED at creation. */
typedef struct {
  int ntypes;
  int sel[DP_MAX_TYPES];
  double rcut;
  double rcut_smth;
  int n_embed;
  int embed[DP_MAX_LAYERS];
  int axis; /* M_< */
  int n_fit;
  int fit[DP_MAX_LAYERS];
  int type_one_side; /* 0: nets N^{a_i,a_j}; 1: nets N^{a_j} */
  int descriptor; /* DP_DESC_*; 0 for an se_e2_a model */
  /* hybrids: the second part */
  double rcut_2, rcut_smth_2;
  int sel_2[DP_MAX_TYPES];
  int n_embed_2;
  int embed_2[DP_MAX_LAYERS];
} dp_model_config;

typedef struct dp_model dp_model;
typedef struct dp_nlist dp_nlist;

/* Create a model on `device` from host FP64 parameters.
 *   params: host, n_params doubles.  Layout: embedding nets in order of net index
 *           (a_i*ntypes + a_j, or a_j if type_one_side; a_j*ntypes + a_k for se_e3), then
 *           (hybrids) the second part's nets in the same way, then fitting nets by type;
 *           per net, layer by layer, W row-major [in][out] then b[out].
 *   precision: DP_PREC_*.  compressed: 1 = replace the embedding nets by quintic
 *           tables (Eq. (compress)) built on the device at creation, over s in
 *           [0, 2] with stride 0.01 on [0, 1.8) and 0.1 on [1.8, 2].
 * Errors: DP_E_ARG (bad config / n_params mismatch), DP_E_OOM, DP_E_CUDA,
 *         DP_E_UNSUPPORTED (e.g. widths beyond the kernels' limits). */
int dp_model_create(const dp_model_config* cfg, const double* params, long n_params, int device, int precision,
                    int compressed, dp_model** out);

/* Same as dp_model_create, reading a weight file: 8-byte magic "DPGBW002", the
 * dp_model_config struct as stored in memory, an int64 n_params, then n_params FP64.
 * Files with magic "DPGBW001" hold the struct up to type_one_side (se_e2_a models). */
int dp_init_model(const char* weight_path, int device, int precision, int compressed, dp_model** out);

int dp_free_model(dp_model* model);

/* Number of FP64 parameters the configuration needs (-1 on a bad config). */
long dp_model_n_params(const dp_model_config* cfg);

/* Build the neighbour list of one frame on the model's device (Sec. III.B.1 order).
 * Per atom i and neighbour type t, the first sel[t] entries of the type-t block hold
 * the neighbours (j, image n) with |r_j + n.h - r_i| < r_c sorted by (r^2, j, n); the
 * rest hold j = -1.  Displacements are evaluated as (r_j + (n0 h0 + n1 h1 + n2 h2)) - r_i
 * left to right in FP64 without fused multiply-add, so lists are bit-reproducible.
 *   n_overflow (host, may be NULL): number of (atom, type) blocks that overflowed sel.
 * Returns DP_OK, or DP_E_SEL_OVERFLOW (list still valid) / DP_E_CAPACITY / DP_E_ARG. */
int dp_build_nlist(dp_model* model, int natoms, const double* coord, const int* type, const double* box,
                   dp_nlist** out, int* n_overflow, void* stream);

/* ---- neighbour list without any allocation ----
 * The paper has no counterpart to this entry point.  It is for callers that cannot
 * allocate device memory at the point where they need a list: an MD engine that owns all
 * device memory and forbids other allocations, or a loop being captured into a CUDA graph.
 * It computes exactly what dp_build_nlist computes (the same bit-exact list, from the same
 * cell binning; the search always runs the per-atom kernel with the full candidate buffer,
 * where dp_build_nlist prefers a cell-centred kernel whose staging buffer is sized per frame)
 * but needs no model object and calls no allocating routine: its cell-list scratch is one
 * static device array of about 13.3 MiB that every GPU loading the library keeps until exit.
 *   cfg: only ntypes, sel and rcut are used (for a hybrid descriptor also rcut_2 and sel_2: the
 *   list is the one its parts read, with the larger cutoff and per type the larger sel).
 *   coord [natoms*3] FP64, type [natoms]: device pointers.  box: host pointer (or NULL for
 *   open boundaries).  nl_j [natoms*Nc], nl_shift [natoms*Nc*3] int32: device pointers the
 *   caller owns, filled exactly as dp_nlist_export fills its host arrays.
 * Limits: natoms <= DP_NOALLOC_MAX_ATOMS, natoms*Nc <= DP_NOALLOC_MAX_SLOTS, cell grid <=
 * DP_NOALLOC_MAX_CELLS cells; larger frames are rejected with DP_E_ARG and a message.
 * The first call on a device looks up the array's device address (one-time set-up, repeated
 * only if the device's context was reset), so make that first call before any stream capture.  All calls on a device share the array:
 * calls that overlap on the GPU race with each other; serialise them (one stream, or
 * events).  Returns as dp_build_nlist; the call synchronises `stream` to read its status. */
#define DP_NOALLOC_MAX_ATOMS 32768
#define DP_NOALLOC_MAX_SLOTS 2097152
#define DP_NOALLOC_MAX_CELLS 32768
int dp_build_nlist_noalloc(const dp_model_config* cfg, int natoms, const double* coord, const int* type,
                           const double* box, int* nl_j, int* nl_shift, int* n_overflow, void* stream);

/* Copy a neighbour list to host arrays nl_j [natoms*Nc] and nl_shift [natoms*Nc*3]. */
int dp_nlist_export(const dp_nlist* nlist, int* nl_j, int* nl_shift);

int dp_free_nlist(dp_nlist* nlist);

/* Energy, forces and virial of one frame.
 *   nlist: a list built by dp_build_nlist from the same coordinates, or NULL to build
 *          one inside the call (the full path).
 *   energy [1], force [natoms*3], virial [9] (row-major Xi_ab), atom_energy [natoms]
 *   (may be NULL).  Outputs may be host or device pointers.
 * Returns DP_OK or a warning/error code as documented above. */
int dp_compute(dp_model* model, dp_nlist* nlist, int natoms, const double* coord, const int* type,
               const double* box, double* energy, double* force, double* virial, double* atom_energy, void* stream);

/* Compressed models: copy the device-built quintic tables (FP64) to host `out`, laid out
 * [net][interval][M][6] with coefficients (a, b, c, d, e, f) of Eq. (compress) for the
 * piece g(t) = a t^5 + ... + f, t = s - x_l.  *n_intervals receives L_c.
 * Returns DP_E_ARG for an uncompressed model. */
int dp_model_export_table(const dp_model* model, double* out, int* n_intervals);

/* ---- tensor-core GEMM used by the fitting net ----
 * C[rows][N] = A[rows][K] . B[K][N] with BF16 operands and FP32 accumulation on the tcgen05
 * tensor cores (the dense layers of Eq. (NN) in the fitting net are this product plus a
 * fused epilogue).  A is [rows][K] row-major, Bt is B transposed ([N][K] row-major), C is
 * [rows][N] row-major FP32; all three are device pointers, K a multiple of 8, both row
 * pitches 16-byte aligned.  Synchronises `stream`.  DP_E_TIMEOUT if a bounded pipeline wait
 * of the kernel gave up (the result is then invalid). */
int dp_gemm_bf16(int rows, int K, int N, const void* A, const void* Bt, float* C, void* stream);

/* ---- tracing (no counterpart in the paper; its TensorBoard profiles play this role) ----
 * dp_profile_enable: when on, every kernel launch of the model's calls is bracketed by CUDA
 * events on the launch stream; per-kernel-name totals are folded in when a call
 * synchronises.  dp_profile_count / dp_profile_read enumerate (name, total ms, launches);
 * dp_profile_reset clears them.  dp_launch_count returns the number of kernels the model's
 * calls have launched since creation or the last reset (counted whether or not timing is on). */
int dp_profile_enable(dp_model* model, int on);
int dp_profile_reset(dp_model* model);
int dp_profile_count(const dp_model* model);
int dp_profile_read(const dp_model* model, int k, char* name, int name_len, double* total_ms, long* count);
long dp_launch_count(const dp_model* model);
/* Tensor-core FLOPs that scope k's kernels issued during the profiled calls (2 x M x N x K of every
 * tcgen05.mma, each pass of a split product counted): counted for the compressed moment
 * contraction ("mom_fwd", "mom_bwd"), whose work depends on the intervals the neighbours occupy;
 * 0 for scopes whose work is a fixed function of the sizes.  DP_E_ARG for a bad index. */
int dp_profile_work(const dp_model* model, int k, double* flop);

/* Energies, forces and virials of several frames, of one or several models, in one call
 * (serving; the batching of frames of Sec. III.B).  The frames keep their own periodic cells and
 * atom counts; their atoms are concatenated.  Consecutive frames of the same model are evaluated
 * together by one pass of that model's kernels (frames of uneven size share every launch); the
 * passes of the models follow each other in stream order.
 *   models [nmodels] (host): the resident models, all on one device.
 *   natoms [nframes] (host): atoms of each frame, in order.
 *   frame_model [nframes] (host): index into models of each frame (may be NULL when nmodels is 1).
 *   coord [sum(natoms)*3] FP64, type [sum(natoms)] int32: host or device, frames concatenated.
 *   boxes [nframes*9] (host): cell rows of every frame (periodic frames only).
 *   energy [nframes], force [sum(natoms)*3], virial [nframes*9], atom_energy [sum(natoms)] or
 *   NULL: host or device.
 * Each frame's result equals dp_compute of its model on that frame alone up to the order of
 * floating-point accumulation.  Returns as dp_compute (the first error ends the call; the
 * warnings DP_E_SEL_OVERFLOW / DP_E_RANGE are returned after all frames are done);
 * DP_E_UNSUPPORTED for boxes == NULL. */
int dp_compute_batch(dp_model** models, int nmodels, int nframes, const int* natoms, const int* frame_model,
                     const double* coord, const int* type, const double* boxes, double* energy, double* force,
                     double* virial, double* atom_energy, void* stream);

/* ---- model deviation of an ensemble (Sec. II.C) ----
 * The n_m = nmodels models (trained on the same data from independent initialisations) evaluate
 * the same frame; their spread estimates the error of the model at that frame:
 *   eps_F,i = sqrt(< |F_i(theta_k) - <F_i>|^2 >),   eps_Xi,ab = (1/N) sqrt(< (Xi_ab(theta_k) - <Xi_ab>)^2 >)
 * with <.> the mean over the models.  nu > 0 selects the relative forms eps_F,i / (|<F_i>| + nu)
 * and eps_Xi,ab / (|<Xi>| + nu) (|<Xi>| the Frobenius norm of the mean virial); nu = 0 the
 * absolute ones.
 *   models [nmodels >= 2] (host), all on one device; coord [natoms*3], type [natoms]: host or
 *   device; box: host [9] or NULL (open boundaries).
 *   devi_f [natoms] (eps_F,i), devi_v [9] (eps_Xi,ab row-major), force_mean [natoms*3] (<F_i>):
 *   host or device, each may be NULL.  stats [6] (host or device): max, mean, min of eps_F,i over
 *   the atoms, then max, mean, min of eps_Xi,ab over the nine components.
 * Everything runs on the GPU in FP64 (the reductions in a fixed order); the models' own
 * precision sets the accuracy of their forces.  Synchronises `stream`.  Returns as dp_compute. */
int dp_model_deviation(dp_model** models, int nmodels, int natoms, const double* coord, const int* type,
                       const double* box, double nu, double* devi_f, double* devi_v, double* stats,
                       double* force_mean, void* stream);

/* ---- training: parameter gradient of an energy + force + virial objective (Sec. II.B) ----
 * The loss of Sec. II.B (Eq. (loss)) weighs energy, force and virial errors (prefactors p_E,
 * p_F, p_Xi).  Its gradient with respect to the parameters needs the derivatives of the force
 * F = -dE/dr and of the virial with respect to every weight: second-order ("double backward")
 * derivatives of E.  This entry point returns, for the model's current parameters,
 *   grad = d/dtheta [ sum_f g_energy[f] E_f + sum_i g_force[i] . F_i + sum_f sum_ab g_virial[f][a][b] Xi_f,ab ]
 * i.e. the vector-Jacobian product of (E, F, Xi) with the cotangents; with g = dL/d(E, F, Xi)
 * it is dL/dtheta for any loss L(E, F, Xi).  All of it runs on the GPU: one tangent pass
 * through the whole path along the pair-displacement tangent (w_j - w_i) + g_virial[f] r_ij
 * (w = g_force; sum g:Xi is minus the derivative of E along that homogeneous deformation),
 * then a reverse pass over the primal and tangent computations.
 *   Frames are passed as for dp_compute_batch (boxes may be NULL only when nframes == 1).
 *   g_energy [nframes], g_force [sum natoms][3] (input atom order), g_virial [nframes][9]
 *   (row-major, or NULL for no virial term; periodic frames only), grad [n_params] in the
 *   parameter layout of dp_model_create; each may be a host or a device pointer.
 * Only uncompressed FP64 and FP32 models (DP_E_UNSUPPORTED otherwise); the arithmetic runs
 * in the model's precision.  Synchronises `stream`.  Returns as dp_compute. */
int dp_param_grad(dp_model* model, int nframes, const int* natoms, const double* coord, const int* type,
                  const double* boxes, const double* g_energy, const double* g_force, const double* g_virial,
                  double* grad, void* stream);

/* Replace the parameters of an uncompressed model in place (a training step's update).
 * params [n_params] FP64, host or device, in the layout of dp_model_create.  Synchronises
 * `stream`.  DP_E_ARG on a size mismatch, DP_E_UNSUPPORTED for compressed models. */
int dp_model_set_params(dp_model* model, const double* params, long n_params, void* stream);

/* Message of the last error raised on the calling thread ("" if none), copied into buf
 * (host, len bytes) and NUL-terminated, truncated to len - 1 characters.  Returns the length of
 * the whole message (as snprintf does), so a caller can size buf; buf may be NULL when len is 0. */
int dp_last_error(char* buf, int len);

/* ---- failure detection self-test (no counterpart in the paper) ----
 * Every wait of the library's tensor-core kernels on an mbarrier (TMA arrivals, MMA completion,
 * the epilogue's hand-backs) is bounded: after a fixed number of polls it records an error,
 * the CTA leaves, and the call returns DP_E_TIMEOUT with the context still usable.  This entry
 * point exercises that mechanism on its own: one CTA initialises an mbarrier that nothing ever
 * arrives at and waits on it through the same bounded-wait routine, with spin_limit polls
 * (<= 0: the limit the kernels use).  No copy or MMA is in flight, so giving up is safe.
 * Returns DP_E_TIMEOUT when the wait gave up (the expected outcome), DP_OK if it completed,
 * DP_E_CUDA on a launch failure.  Synchronises `stream`. */
int dp_wait_selftest(long spin_limit, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DPGB_H */
