/*
 * qt.h -- C ABI of libqt, the GB300 (sm_103a) library for the forward step of
 * the Quantization Tree algorithm and its backward induction.
 *
 * Method: G. Pages and B. Wilbertz, "GPGPUs in computational finance: Massive
 * parallel computing for American style options", arXiv:1101.3228.
 *   Sec. 2        quantization grids Gamma_k, Voronoi cells, nearest-neighbour
 *                 projection, transition probabilities (eq. (defPi)), the BDP
 *                 recursion on the tree;
 *   Sec. 3        the Gaussian 2-factor model, Prop. 1 (AR(1) form
 *                 X_{k+1} = A_k X_k + T_k eps_k), Algorithm I;
 *   Sec. 3.1-3.3  random numbers, nearest-neighbour search, counter updates;
 *   Sec. 4        Algorithm III: every layer k draws M pairs (X_k, eps_k)
 *                 independently, i = NN(X_k, Gamma_k),
 *                 j = NN(A_k X_k + T_k eps_k, Gamma_{k+1}), counts p^k_ij,
 *                 then pi^k_ij = p^k_ij / p^k_i.
 *
 * Conventions common to every entry point
 *   - Status: every function returns a qt_status; 0 is success.  Errors never
 *     unwind across the ABI.  qt_last_error() returns a message for the last
 *     failing call on that context.
 *   - Asynchrony: work is enqueued on the caller's CUDA stream (a cudaStream_t
 *     passed as void*; NULL is the legacy default stream).  Functions that
 *     return host results (qt_price, qt_get_status, and any call given a
 *     non-NULL qt_stats*) synchronise that stream before returning.
 *   - Ownership: every pointer argument is owned by the caller.  The library
 *     owns only the context and the workspace it allocates inside it.  "dev"
 *     marks device pointers, "host" marks host pointers; qt_price also accepts
 *     host memory where it says so.
 *   - Layout: all arrays are C-contiguous, row-major.  Grids of all layers are
 *     concatenated: layer k occupies points [off_k, off_k + N_k) of a
 *     [sum_k N_k][d] FP64 array.  Count matrices are concatenated the same way:
 *     layer k is an [N_k][N_{k+1}] block at entry offset sum_{q<k} N_q N_{q+1}.
 *   - Exactness contract: the cell of a point z in Gamma is
 *     argmin_i D64(z, x_i), D64 = sum_l (z_l - x_il)^2 accumulated left to
 *     right in IEEE binary64 with round-to-nearest and no fused multiply-add;
 *     equal distances go to the lowest index.  Every search form returns this
 *     cell for every sample ("certified"), whatever precision it screens in.
 *   - Sampler: Philox4x32-10 (Salmon et al., SC'11) with key (seed_lo, seed_hi)
 *     and counter (m_lo, m_hi, k, r) for sample m of layer k and call r;
 *     Box-Muller normals from uniforms u = (2 floor(w/2^9) + 1) 2^-24 (FP32)
 *     or from two words (FP64), with ln, sin and cos evaluated by fixed
 *     series in correctly rounded arithmetic; z = normals [0,d),
 *     eps = normals [d,2d); X_k = m_k + L_k z; Y = A_k X_k + b_k + T_k eps,
 *     each product and sum rounded in order in the sample precision.  The
 *     samples are therefore the same bits on any IEEE machine.
 */
#ifndef QT_H
#define QT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QT_API __attribute__((visibility("default")))
#else
#define QT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qt_status;
#define QT_OK 0
#define QT_EINVAL 1          /* an argument is out of range or inconsistent            */
#define QT_ENOMEM 2          /* a device or host allocation failed                     */
#define QT_ECUDA 3           /* a CUDA runtime call failed (message has the CUDA error) */
#define QT_ETIMEOUT 4        /* a bounded device wait ran out; results are not valid    */
#define QT_EUNSUPPORTED 5    /* the request needs a form or size this build lacks       */
#define QT_EDEVICE 6         /* a kernel reported an internal inconsistency             */

/* search forms (qt_options.form) */
#define QT_FORM_AUTO 0        /* library picks the fastest certified form: TC_RECHECK for
                                 3 <= d <= 10, F32_RECHECK otherwise                      */
#define QT_FORM_PLAIN_F64 1   /* brute force, exact FP64 distances                       */
#define QT_FORM_F32_RECHECK 2 /* FP32 brute-force screen, FP64 recheck of near ties      */
#define QT_FORM_TC_RECHECK 3  /* tensor-core (tcgen05) screen, FP64 recheck              */
#define QT_FORM_ROUTER_CERT 4 /* learned start cell + Elkan certificate, brute fallback  */

/* sample precision (qt_options.sample_prec) */
#define QT_PREC_F64 0
#define QT_PREC_F32 1

/* count element type (qt_options.counts_type) */
#define QT_COUNTS_I64 0
#define QT_COUNTS_U32 1

/* qt_options.flags */
#define QT_FLAG_NO_GRAPH 1u   /* launch kernels directly instead of replaying a CUDA graph */
#define QT_FLAG_NO_TUNE 2u    /* skip the autotuner, use the built-in tile choice            */
#define QT_FLAG_SMEM_HIST 4u  /* force the shared-memory privatised histogram                */
#define QT_FLAG_GLOBAL_HIST 8u /* force direct L2 atomics for the counts                     */
#define QT_FLAG_FUSED_BACKWARD 16u /* qt_price: layer pairs in reverse order, each pair's counts
                                    folded into V at once (one pair's counts in memory)       */

/* grid-building methods (qt_build_grids) */
#define QT_GRID_LLOYD1D 1     /* d = 1: stationary quantizer of N(0,1) (Newton on Lloyd's map) */
#define QT_GRID_PRODUCT 2     /* product of 1-d stationary quantizers                          */
#define QT_GRID_KMEANS 3      /* sample Lloyd (k-means) on seeded N(0, I_d) draws              */

typedef struct qt_ctx qt_ctx;

/* The Markov chain of Prop. 1 on layers k = 0..n (host arrays, FP64).
 *   N [n+1]        grid sizes N_k >= 1 (N_0 = 1 when X_0 is deterministic)
 *   A [n][d][d]    AR(1) matrices A_k
 *   b [n][d]       drifts b_k (zero for the OU model of Sec. 3)
 *   T [n][d][d]    innovation factors T_k, read as lower triangular
 *   m [n+1][d]     mean of X_k
 *   L [n+1][d][d]  lower-triangular factor of Cov(X_k), read as lower triangular
 * 1 <= d <= 16, 1 <= n <= 65535.                                                 */
typedef struct {
    int32_t d;
    int32_t n;
    const int64_t* N;
    const double* A;
    const double* b;
    const double* T;
    const double* m;
    const double* L;
} qt_model;

typedef struct {
    int32_t form;          /* QT_FORM_*                                                    */
    int32_t sample_prec;   /* QT_PREC_*                                                    */
    int32_t counts_type;   /* QT_COUNTS_* (element type of the counts array)               */
    uint32_t flags;        /* QT_FLAG_*                                                    */
    int64_t spin_budget;   /* bound of every device wait, in microseconds of the GPU's global
                              timer; 0 = library default (10 s); negative = give up at once
                              (tests of the timeout path)                                  */
    const void* router;    /* qt_router* for QT_FORM_ROUTER_CERT, else NULL                */
    int32_t tile_samples_per_thread; /* 0 = autotuned                                       */
    int32_t tc_chunk_items; /* tensor-core form: most work items (128 samples each) per kernel
                              launch; 0 = the whole step in one launch (draw-pass layout:
                              as many as 2 GiB of drawn samples hold)                      */
    int32_t tc_draw;       /* tensor-core form: where the samples are drawn.  0 = autotuned
                              (both timed once per dimension class), 1 = a separate draw
                              pass writes them to device memory before each screen launch,
                              2 = the screen kernel draws them itself (one launch, no
                              device-memory hand-off)                                     */
    int32_t reserved[1];
} qt_options;

/* Optional per-sample record: sample t of layer k is m = t * stride, t < count.
 * X, Y: dev FP64 [n][count][d]; i, j: dev int32 [n][count] (-1 where m >= M). */
typedef struct {
    int64_t count;
    int64_t stride;
    double* X;
    double* Y;
    int32_t* i;
    int32_t* j;
} qt_dump;

/* Filled by calls given a non-NULL qt_stats* (the call then synchronises). */
typedef struct {
    int64_t samples;        /* sample pairs processed (n * M)                        */
    int64_t rechecks;       /* FP64 re-evaluations of an uncertain screened search   */
    int64_t searches;       /* nearest-cell searches (2 per sample pair)              */
    int64_t candidates;     /* screened candidate distances (router form)             */
    int32_t form_used;      /* QT_FORM_* actually run                                 */
    int32_t device_status;  /* qt_status reported by the kernels                      */
    double ms;              /* device time of the forward step, if measured, else 0   */
    int64_t diag[3];        /* tensor-core form: uncertified picks by cause (FP32 bound
                               inside the re-scored chunks, tensor-core bound outside
                               them, index or FP16 range)                              */
    int32_t launches;       /* kernels the forward step launched (preparation, draw
                               passes, screens)                                        */
    int32_t tc_draw;        /* tensor-core form: sample-draw layout run (1 = draw pass,
                               2 = inside the screen kernel), else 0                   */
} qt_stats;

/* Context: one per device.  device = CUDA ordinal.  Not thread safe; use one
 * context per host thread.  qt_destroy frees everything the context owns.    */
QT_API qt_status qt_create(qt_ctx** ctx, int32_t device);
QT_API qt_status qt_destroy(qt_ctx* ctx);
QT_API const char* qt_last_error(const qt_ctx* ctx);
QT_API const char* qt_status_string(qt_status s);
/* Default options: AUTO form, FP32 samples, int64 counts, autotuned tiles. */
QT_API void qt_default_options(qt_options* opts);

/* Grids for every layer (Sec. 2: grids that minimise the quadratic error of
 * eq. (Qerr); the paper's precomputed optimal Gaussian grids are replaced by
 * stationary quantizers built here).  Layer k gets m_k + L_k g for a base grid
 * g of N(0, I_d) with N_k points.  method = QT_GRID_*; samples and iters are
 * used by QT_GRID_KMEANS (training draws, Lloyd iterations); tol is the Newton
 * tolerance of the 1-d quantizer.  grids: dev FP64 [sum_k N_k][d], written.   */
QT_API qt_status qt_build_grids(qt_ctx* ctx, const qt_model* model, int32_t method, int64_t samples,
                         int32_t iters, double tol, uint64_t seed, double* grids, void* stream);

/* Algorithm III (Sec. 4): for k = 0..n-1 and m = 0..M-1 draw (X_k, eps_k),
 * find i = NN(X_k, Gamma_k) and j = NN(A_k X_k + b_k + T_k eps_k, Gamma_{k+1})
 * and add 1 to p^k_ij.  All layers run in one persistent launch.
 *   grids  dev FP64 [sum_k N_k][d]
 *   counts dev [sum_k N_k N_{k+1}] of opts->counts_type, OVERWRITTEN (zeroed
 *          first); p^k_i = sum_j p^k_ij is not stored (row sums).
 *   M      samples per layer, 1 <= M < 2^32
 *   dump   optional per-sample record (may be NULL); stats optional.        */
QT_API qt_status qt_transitions(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M,
                         uint64_t seed, const qt_options* opts, void* counts, const qt_dump* dump,
                         qt_stats* stats, void* stream);

/* Algorithm II (Sec. 3, Algorithms I and II): the path-wise estimator.  Every
 * path m runs through all layers: X_0 = m_0 + L_0 z with z = normals [0, d)
 * of stream (m, 0); for k = 0..n-1, eps_k = normals [d, 2d) of stream (m, k),
 * X_{k+1} = b_k + A_k X_k + S_k(X_k) T_k eps_k, j = NN(X_{k+1}, Gamma_{k+1})
 * and p^k_ij += 1 with i the cell of X_k.  One search per path and layer
 * (Algorithm III makes two), sequential in k; the counts estimate the same
 * pi^k_ij, and the first step is Algorithm III's layer-0 pair.
 *   euler  NULL: the AR(1) chain of Prop. 1 (S_k = I).  Otherwise the Euler
 *          step of a square-root diffusion, a chain that is not AR(1):
 *          S_k = diag(s_kl), s_kl(x) = sqrt(max(alpha_kl + beta_kl x_l, 0)),
 *          alpha, beta host FP64 [n][d].  In the sample precision, each
 *          operation rounded in the order s_l = sqrt(max(alpha_l + beta_l*x_l, 0)),
 *          t_lq = s_l*T_lq, acc = b_l, acc += A_lq*x_q (q ascending),
 *          acc += t_lq*eps_q (q <= l).
 *   opts   form QT_FORM_AUTO or QT_FORM_F32_RECHECK (FP32 screen with the exact
 *          recheck: cells exact under the library contract); FP32 or FP64
 *          samples.  Grids of any size (streamed through shared memory in
 *          segments when they exceed half of it).
 *   counts, dump, stats as in qt_transitions (dump row k holds X_k, X_{k+1}
 *          and their cells); model->m and L are read for layer 0 only.      */
typedef struct {
    const double* alpha;   /* host FP64 [n][d] */
    const double* beta;    /* host FP64 [n][d] */
} qt_euler;

QT_API qt_status qt_transitions_pathwise(qt_ctx* ctx, const qt_model* model, const qt_euler* euler,
                                         const double* grids, int64_t M, uint64_t seed, const qt_options* opts,
                                         void* counts, const qt_dump* dump, qt_stats* stats, void* stream);

/* Counting step of Algorithm III on caller-supplied samples (one layer pair):
 * counts[NA][NB] (dev, opts->counts_type) is OVERWRITTEN with
 * #{t : NN(X_t, gA) = i, NN(Y_t, gB) = j}.  gA dev FP64 [NA][d], gB [NB][d],
 * X, Y dev FP64 [M][d] (finite values).  ii/jj (dev int32 [M]) receive the
 * cells when non-NULL.                                                         */
QT_API qt_status qt_counts_from_samples(qt_ctx* ctx, int32_t d, const double* gA, int64_t NA,
                                 const double* gB, int64_t NB, const double* X, const double* Y,
                                 int64_t M, const qt_options* opts, void* counts, int32_t* ii,
                                 int32_t* jj, qt_stats* stats, void* stream);

/* BDP recursion on the tree (Sec. 2): V_n = phi_n and, for k = n-1..0,
 * V_k(i) = max(phi_k(i), sum_j pi^k_ij V_{k+1}(j)) with pi^k_ij = p^k_ij / p^k_i
 * (Algorithm III's normalisation).  A row with p^k_i = 0 has no continuation:
 * V_k(i) = phi_k(i).  The continuation is evaluated as
 * (sum_j p^k_ij V_{k+1}(j)) / p^k_i in FP64, j summed in lanes j mod 32 and
 * combined by a fixed butterfly, so results are bitwise reproducible.
 *   N      host int64 [n+1]
 *   counts dev, counts_type elements, concatenated as in qt_transitions
 *   phi, V dev FP64 [sum_k N_k] (V written)                                    */
QT_API qt_status qt_backward(qt_ctx* ctx, int32_t n, const int64_t* N, const void* counts,
                      int32_t counts_type, const double* phi, double* V, void* stream);

/* Swing option on the tree (Sec. 2, eq. (stochCtrl) and the bang-bang BDP that
 * follows it): controls x_k in {0, 1} at dates k = 0..n-1, payoff x_k v_k(X_k),
 * global constraint sum_k x_k in [Qmin, Qmax].  The paper leaves the
 * admissible set I_Q and the transition chi of the consumption state Q to its
 * reference; read here as chi(Q, x) = Q + x, and x admissible at (k, Q) when the
 * consumption can still end inside [Qmin, Qmax]: F(k+1, Q + x) with
 * F(k, Q) = (Q <= Qmax and Q + n - k >= Qmin).
 *   P_n(., Q) = 0 where F(n, Q), -inf elsewhere;
 *   P_k(i, Q) = max over admissible x of x v_k(i) + C_k(i, Q + x), -inf where
 *               none is admissible;  C_k(i, Q') = (sum_j p^k_ij P_{k+1}(j, Q')) / p^k_i
 *               in the fixed order of qt_backward (0 for an empty row).
 * Qmax = 1, Qmin = 0 is the Bermudan of qt_backward with phi_n = 0, bit for bit.
 *   N       host int64 [n+1];  counts dev, as in qt_backward
 *   v       dev FP64 [sum_k N_k] payoff values (layer n unused)
 *   P       dev FP64 [(Qmax + 1) * sum_k N_k], written: layer k is a Q-major
 *           [Qmax + 1][N_k] block at offset (Qmax + 1) * sum_{q<k} N_q
 *   price   host, optional: P_0(x_0, 0) if N_0 = 1, else sum_i (p^0_i / M) P_0(i, 0);
 *           given, the call synchronises the stream.
 * 0 <= Qmin <= min(Qmax, n), Qmax <= 2^20; QT_EINVAL otherwise.               */
QT_API qt_status qt_swing(qt_ctx* ctx, int32_t n, const int64_t* N, const void* counts, int32_t counts_type,
                          const double* v, int32_t Qmin, int32_t Qmax, double* P, double* price, void* stream);

/* Forward step + backward induction + root value: the option price V^_0.
 * If N_0 = 1 the price is V_0(0); otherwise sum_i (p^0_i / M) V_0(i).
 * grids and phi may be host or dev pointers (FP64 [sum_k N_k][d] and
 * [sum_k N_k]); price is a host double.  Synchronises the stream.             */
QT_API qt_status qt_price(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M,
                   uint64_t seed, const qt_options* opts, const double* phi, double* price,
                   qt_stats* stats, void* stream);

/* Synchronise the stream and return the device status of the last forward
 * call on this context (QT_OK, QT_ETIMEOUT or QT_EDEVICE).                    */
QT_API qt_status qt_get_status(qt_ctx* ctx, void* stream, qt_stats* stats);

/* Device bytes the context will allocate for a qt_transitions call of this
 * shape (descriptor tables, prepared grids, status words).                   */
QT_API qt_status qt_transitions_workspace(const qt_model* model, const qt_options* opts, size_t* bytes);

/* ------------------------------------------------------------------------
 * Learned router + Elkan certificate (search form QT_FORM_ROUTER_CERT).
 * No paper counterpart for the network itself; the certificate restates the
 * triangle inequality on the Voronoi cells of Sec. 2: if |x - c_i0| = r then the
 * nearest cell j of x satisfies |c_i0 - c_j| <= 2r, so scanning the points of
 * Gamma_k sorted by distance to c_i0 until that distance exceeds r + r* (r* the
 * best distance found so far) finds the exact cell from any start cell i0.
 * The router (an MLP d -> 64 -> 64 -> 64, ReLU, on whitened coordinates
 * L_k^{-1}(x - m_k)) predicts which of 64 buckets (a k-means partition of the
 * grid points) holds the cell; the start cell is the nearest member of the two
 * most likely buckets.  Training runs in FP32 on the CUDA cores; the search
 * evaluates the network on the tensor cores (FP16 operands, FP32 accumulators,
 * 128 samples per tile).  A wrong prediction, or a rounding of the FP16
 * inference, costs time, never exactness.
 * Requires N_k equal for all k >= 1 (one bucket partition serves every layer),
 * 64 <= N_k <= 8192 and d <= 16.                                              */
typedef struct qt_router qt_router;

typedef struct {
    int64_t train_samples;   /* labelled (sample, exact cell) pairs; 0 = 10^6            */
    int32_t train_layers;    /* layers the pairs are drawn from (evenly spaced); 0 = 8    */
    int32_t epochs;          /* passes over the pairs; 0 = 8                               */
    int32_t batch;           /* minibatch; 0 = 4096                                        */
    int32_t neighbours;      /* sorted neighbours kept per grid point (Elkan list); 0 = 1024,
                                at most N_k - 1                                            */
    float lr;                /* Adam step; 0 = 3e-3                                        */
    int32_t untrained;       /* 1: keep the seeded initial weights (for comparisons)       */
    int32_t reserved[3];
} qt_router_config;

typedef struct {
    int64_t params;          /* number of FP32 parameters                                  */
    int32_t d, buckets, hidden, neighbours;
    double train_loss;       /* mean cross-entropy of the last epoch                       */
    double train_accuracy;   /* top-1 bucket accuracy on the training pairs (last epoch)   */
    double build_ms;         /* wall time of qt_router_train                               */
} qt_router_info;

/* Train a router for `model` and `grids` (dev FP64, concatenated as in
 * qt_transitions): draws cfg->train_samples pairs (X_k, exact cell of X_k in
 * Gamma_k) with the library's own sampler and search, trains the MLP with the
 * library's own forward, backward and Adam kernels, and builds the bucket and
 * neighbour tables of every grid.  The router is bound to these grids: a
 * qt_transitions call with other grid values returns QT_EINVAL.  *out is owned
 * by the caller (qt_router_destroy).  Synchronises the stream.                */
QT_API qt_status qt_router_train(qt_ctx* ctx, const qt_model* model, const double* grids, const qt_router_config* cfg,
                                 uint64_t seed, qt_router** out, void* stream);
QT_API qt_status qt_router_destroy(qt_router* router);
QT_API qt_status qt_router_get_info(const qt_router* router, qt_router_info* info);

/* Copy the MLP parameters (FP32, packed W1[64][d], b1[64], W2[64][64], b2[64],
 * W3[64][64], b3[64]) to host memory `out` (count floats) or set them from
 * host memory `in`; count must equal info.params.                             */
QT_API qt_status qt_router_get_params(const qt_router* router, float* out, int64_t count);
QT_API qt_status qt_router_set_params(qt_router* router, const float* in, int64_t count);

/* Mean cross-entropy over a batch and its gradient with respect to every
 * parameter, from the library's own kernels (used to check them): z dev FP32
 * [B][d], labels dev int32 [B] in [0, 64), grad dev FP32 [params] (written),
 * loss host.  Synchronises the stream.                                        */
QT_API qt_status qt_router_loss_grad(qt_ctx* ctx, const qt_router* router, const float* z, const int32_t* labels,
                                     int64_t B, float* grad, double* loss, void* stream);

/* Allocation-free counting step, for callers that cannot allocate device
 * memory (a host application whose allocator has reserved the device memory,
 * a plug-in that may not own device memory, or a latency-bound loop that cannot
 * afford the implicit synchronisation of cudaMalloc/cudaFree).  The paper has
 * no counterpart: this is a packaging variant of qt_counts_from_samples.
 *
 * Same arguments and result as qt_counts_from_samples with the FP32 screen and
 * FP64 recheck (counts OVERWRITTEN, cells optional), on the CURRENT device,
 * without a context: the scratch (status and queue words, descriptors, a copy
 * of both grids, their screened records) is a fixed array inside the library,
 * one per device, kept until the process exits.  It calls no allocation
 * routine.  The first call on a device looks up the array's device address and
 * two device attributes and keeps them for the life of the process; make that
 * first call before any stream capture, and do not call this entry point on a
 * device after cudaDeviceReset (the kept address would be stale).  Every call
 * reuses the same
 * array, so calls that overlap on the GPU (two streams, two host threads)
 * race: serialise them.  The call synchronises `stream` and returns the
 * kernels' status.
 * Limits: 1 <= d <= 16, NA + NB <= QT_NOALLOC_MAX_POINTS, and the screened
 * records of both grids must fit one CTA's shared memory; otherwise QT_EINVAL
 * is returned before any work is enqueued.                                    */
#define QT_NOALLOC_MAX_POINTS 4096
QT_API qt_status qt_counts_from_samples_noalloc(int32_t d, const double* gA, int64_t NA, const double* gB,
                                                int64_t NB, const double* X, const double* Y, int64_t M,
                                                int32_t counts_type, void* counts, int32_t* ii, int32_t* jj,
                                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QT_H */
