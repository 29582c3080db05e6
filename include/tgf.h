/*
 * tgf.h -- C ABI of libtgf: the twisted Wilson flow of SU(3) link fields on a GB300 (sm_103a).
 *
 * The library integrates the Wilson flow dV/dt = Z(V) V, Z = -g0^2 dS_W, of the
 * twisted Wilson action S_W = 3b sum_n sum_{mu!=nu} Tr[1 - Z*_{mu nu}(n) P_{mu nu}(n)]
 * (arXiv:2107.03747, Sec. 3.1) with Luscher's third-order Runge-Kutta scheme
 * (JHEP 08 (2010) 071, cited in Sec. 1), and measures along the flow the clover
 * energy density E(t) and topological charge Q(t) (Sec. 3.1, eqs. gmunu and qlatt)
 * and the average twisted plaquette.  Host helpers give the lattice
 * normalisation N(c, Lt) (eq. latt_norm) and lambda_TGF (eq. lambdat_latt).
 *
 * Memory.  The stateless calls allocate no device memory.  Every device buffer
 * is owned by the caller (for example a torch tensor) and passed as a plain
 * pointer; sizes come from the tgf_*_bytes queries.  Only the context calls
 * (tgf_create and the tgf_ctx_* family) allocate, and they own what they
 * allocate.  Device pointers must be
 * 256-byte aligned (cudaMalloc and torch allocations are).  Host pointers are
 * read or written only during the call unless stated otherwise.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Device work is enqueued on it and the call returns without
 * synchronising unless stated otherwise.
 *
 * Errors.  Every call returns a tgf_status; nothing is thrown across the ABI.
 * On failure tgf_last_error() returns a message (thread-local, valid until the
 * next failing call on the same thread).  Invalid arguments are rejected before
 * any device work is enqueued.  Kernels never wait on a flag, a peer or a
 * timer, so no call can time out; a record that comes out non-finite (NaN or
 * infinite links, or an overflow) is noted in a device word that TGF_SYNC calls
 * and tgf_kernel_status() turn into TGF_EKERNEL.
 *
 * Fault injection (tests of error handling; nothing faults on the GPU): the
 * environment variable TGF_FAULT, read at every call, makes tgf_create fail
 * with TGF_ENOMEM before allocating (=alloc), makes tgf_upload and
 * tgf_set_links plant a NaN in the device copy of the first real they upload
 * (=nan; the caller's buffer is untouched), or makes the argument checks of
 * tgf_stage, tgf_measure, tgf_measure_slices and tgf_flow fail with TGF_EINVAL
 * (=badarg).
 *
 * Threading and device state.  Calls on different streams, or from different
 * host threads, share no mutable state except the cache of captured flow
 * graphs (guarded by a lock), the device word of non-finite records (one per
 * device) and tgf_measure_noalloc's fixed array (one per device).  The graph
 * cache and that array's address are per CUDA context: after cudaDeviceReset
 * the library must not be used again in the same process.
 *
 * Lattices.  A batch is `ncfg` (1..TGF_MAX_CFG) configurations, each with its
 * own tgf_lattice: extents L[0..3] (x0 fastest; directions 0, 1 are the short
 * twisted plane of the l x l x 3l x 3l box, 2, 3 the long periodic ones) and
 * the antisymmetric twist tensor n_{mu nu} mod 3 given by its six upper
 * entries.  The extents must be the paper's box (l, l, 3l, 3l) (Sec. 3.1; for
 * the SU(N) calls (l, l, Nl, Nl)), else the call returns TGF_EINVAL, unless the
 * configuration's flags hold TGF_ANY_EXTENTS, which admits any extents >= 2
 * (tests of ragged and odd boxes).  The centre factor Z_{mu nu}(n) = exp(2 pi i n_{mu nu}/3)
 * sits on the plaquettes whose corner has x_mu = x_nu = 0 (the 0-based reading
 * of the paper's x_1 = x_2 = 1) and is 1 elsewhere.
 *
 * Canonical layout (host and device "canonical" buffers): per configuration
 * V = L0 L1 L2 L3 sites x 4 directions x 3 x 3 complex doubles, ordered
 * [x3][x2][x1][x0][mu][row][col][re,im]; configurations follow each other.
 *
 * Device storage layout (opaque to callers, described for profiling): per
 * configuration, per direction, 16-byte-vector planes of Vp = V rounded up to
 * a multiple of 32 sites -- FP64: nine double2 planes (matrix entries);
 * FP32: four float4 planes (entries 0-7) and one float2 plane (entry 8);
 * FP32_R12: three float4 planes holding rows 0 and 1, row 2 being rebuilt on
 * every load as conj(row0 x row1).  The su(3) accumulator X of the RK3 scheme
 * holds 8 reals per link in the working precision.
 */
#ifndef TGF_H
#define TGF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TGF_OK = 0,
    TGF_EINVAL = 1,   /* bad argument: extents, twist, sizes, pointers, eps, t_end   */
    TGF_ENOMEM = 2,   /* tgf_create could not allocate its device memory              */
    TGF_ECUDA = 3,    /* a CUDA runtime call failed (message in tgf_last_error)      */
    TGF_EKERNEL = 4,  /* a measured record is not finite (TGF_SYNC calls, tgf_kernel_status) */
    TGF_ESTATE = 6,   /* no configuration survived the |Q| < 1/2 cut                  */
    TGF_EIO = 7       /* checkpoint file missing, unreadable, truncated or corrupted  */
} tgf_status;

typedef enum {
    TGF_FP64 = 0,     /* links, staples, exponential, X in double                     */
    TGF_FP32 = 1,     /* links (18 reals), staples, exponential, X in float; sums FP64 */
    TGF_FP32_R12 = 2  /* as TGF_FP32 with links stored as two rows (12 reals)          */
} tgf_precision;

#define TGF_MAX_CFG 256

/* Flags of tgf_measure / tgf_flow. */
#define TGF_CLOVER_TRACELESS 1u   /* subtract tr(G)/3 from the clover G (eq. gmunu has no projection) */
#define TGF_NO_GRAPH 2u           /* tgf_flow: launch kernels directly instead of one CUDA graph      */
#define TGF_SYNC 4u               /* tgf_measure / tgf_flow: synchronise `stream`, then return
                                     TGF_EKERNEL if a record written on this device since the last
                                     such check is not finite                                       */
/* Launch tuning of tgf_flow (results are bitwise the same for every setting; the tuner of the
 * Python package times them per workload): TGF_TUNE_GRID(k), k = 1..15, launches the stage
 * kernels as a persistent grid of k x (number of SMs) x (resident blocks per SM: 4 in FP32,
 * 2 in FP64) that loops over the tiles, instead of one block per tile (k = 0);
 * TGF_TUNE_SIZE_ORDER orders the configurations of each launch by size, largest first. */
#define TGF_TUNE_GRID(k) (((unsigned)(k) & 0xFu) << 8)
#define TGF_TUNE_SIZE_ORDER (1u << 12)
/* TGF_TUNE_TILE(t): launch tile of the FP32 forms' stage kernels -- 0: 32 consecutive sites per
 * block, one warp per direction, 4 blocks per SM; 1: 64 sites per block (two warps per
 * direction); 2: 32 sites per block as a 4 x 2 x 2 x 2 hypercube (where L0 % 4 == 0 and L1, L2,
 * L3 are even; consecutive sites otherwise); 3: as 0, with the forward-staple corners
 * U_b(n+a) U_a(n+b)^+ of the unmeasured stages formed once per pair of direction warps and passed
 * through shared memory; 4: as 0 with 5 blocks per SM in the unmeasured stages (tighter register
 * cap).  Tiles 0, 1, 2, 4 give bitwise the same flow, 3 the same up to rounding.  Ignored in FP64. */
#define TGF_TUNE_TILE(t) (((unsigned)(t) & 0x7u) << 13)

typedef struct {
    int L[4];        /* extents, x0 fastest                                          */
    int twist[6];    /* n_01, n_02, n_03, n_12, n_13, n_23 (any integers, taken mod 3) */
    unsigned flags;  /* 0, or TGF_ANY_EXTENTS                                        */
} tgf_lattice;

/* tgf_lattice.flags: accept any extents >= 2 instead of only the box (l, l, 3l, 3l). */
#define TGF_ANY_EXTENTS 1u

/* One measurement of one configuration (Sec. 3.1).
 *   t  flow time
 *   E  (1/V) sum_n 1/2 Tr[G_{mu nu} G_{mu nu}]                       clover energy density
 *   Q  1/(16 pi^2) sum_n Tr[G_{mu nu} Gt_{mu nu}]                    clover topological charge
 *   P  (1/(6V)) sum_n sum_{mu<nu} 1/3 Re Tr[Z*_{mu nu} P_{mu nu}]   average twisted plaquette
 *   S  sum_n sum_{mu<nu} Re Tr[1 - Z* P] = g0^2 S_W / 2              reduced twisted action   */
typedef struct {
    double t, E, Q, P, S;
} tgf_obs;

/* ---- sizes ---------------------------------------------------------------------------- */

/* Bytes of device link storage for the batch in precision `prec` (see layout above). */
tgf_status tgf_links_bytes(int prec, const tgf_lattice *lat, int ncfg, size_t *bytes);
/* Bytes of the RK3 accumulator X (8 reals per link in the working precision). */
tgf_status tgf_accum_bytes(int prec, const tgf_lattice *lat, int ncfg, size_t *bytes);
/* Bytes of the scratch buffer that tgf_measure and tgf_flow use: per-block FP64 partial sums
 * and, per site, the two halves of the clover's anti-Hermitian part for the six planes plus the
 * six twisted plaquette traces (114 reals per site in the working precision). */
tgf_status tgf_scratch_bytes(int prec, const tgf_lattice *lat, int ncfg, size_t *bytes);
/* Bytes of one configuration's canonical FP64 field: V * 4 * 9 * 16. */
tgf_status tgf_canonical_bytes(const tgf_lattice *lat, size_t *bytes);

/* ---- layout conversion (Sec. 3.1 links U_mu(n)) --------------------------------------- */

/* Canonical FP64 device buffer (all configurations) -> device storage `links`. FP32 forms
 * round to nearest; FP32_R12 keeps rows 0 and 1. */
tgf_status tgf_pack(int prec, const tgf_lattice *lat, int ncfg, const double *canon_dev,
                    void *links, void *stream);
/* Device storage -> canonical FP64 device buffer (FP32_R12 rebuilds row 2). */
tgf_status tgf_unpack(int prec, const tgf_lattice *lat, int ncfg, const void *links,
                      double *canon_dev, void *stream);
/* Host canonical buffer -> device storage, one configuration at a time through the caller's
 * device staging buffer of at least max-over-configurations tgf_canonical_bytes.  The host
 * buffer should be pinned for the copies to be asynchronous; it must stay valid until the
 * stream reaches this point. */
tgf_status tgf_upload(int prec, const tgf_lattice *lat, int ncfg, const double *canon_host,
                      double *staging_dev, size_t staging_bytes, void *links, void *stream);
/* Device storage -> host canonical buffer through the staging buffer; synchronises `stream`. */
tgf_status tgf_download(int prec, const tgf_lattice *lat, int ncfg, const void *links,
                        double *staging_dev, size_t staging_bytes, double *canon_host, void *stream);

/* ---- the hot path ----------------------------------------------------------------------- */

/* One stage s = 1, 2, 3 of the low-storage RK3 step of size eps for every link of the batch:
 * Z = -P_ta(U_mu Sigma_mu) from the twisted staples of `w_in`; then
 *   s=1: X = eps Z/4;   s=2: X = 8/9 eps Z - 17/9 X;   s=3: X = 3/4 eps Z - X;
 * and w_out = exp(X) w_in (exact SU(3) exponential).  The three stages equal Luscher's
 * W1 = e^{Z0/4} W0, W2 = e^{8/9 Z1 - 17/36 Z0} W1, W3 = e^{3/4 Z2 - 8/9 Z1 + 17/36 Z0} W2.
 * w_in and w_out must not overlap.  reunit != 0 (stage 3, FP32 forms) re-projects w_out onto
 * SU(3) by Gram-Schmidt in FP64 before storing.  flags: 0 or TGF_TUNE_TILE(t), the launch tile of
 * the FP32 forms (as in tgf_flow). */
tgf_status tgf_stage(int prec, const tgf_lattice *lat, int ncfg, const void *w_in, void *w_out,
                     void *accum, int stage, double eps, int reunit, unsigned flags, void *stream);

/* Measure every configuration of `links` at flow time t: obs_dev[c * obs_stride + rec] receives
 * {t, E, Q, P, S} of configuration c.  `scratch` holds the per-block partial sums (size from
 * tgf_scratch_bytes).  Sums are taken in FP64 in a fixed order (bitwise reproducible). */
tgf_status tgf_measure(int prec, const tgf_lattice *lat, int ncfg, const void *links,
                       double *scratch, size_t scratch_bytes, tgf_obs *obs_dev, size_t obs_stride,
                       int rec, double t, unsigned flags, void *stream);

/* Synchronise `stream`, then return TGF_EKERNEL (with the configuration and record in the
 * message) if a record written on the current device since the last check is not finite, and
 * clear the note.  The paper has no counterpart: this is the library's failure report. */
tgf_status tgf_kernel_status(void *stream);

/* tgf_measure for callers that cannot allocate device memory: the same measurement, with the
 * scratch held in a fixed device array inside the library instead of a caller buffer.  The
 * paper has no counterpart; it serves code that may not call cudaMalloc, such as a plug-in
 * whose host application owns all device memory and passes in only inputs and outputs, or a
 * latency-critical loop that must avoid cudaMalloc's implicit device synchronisation.  The
 * caller still passes the links and obs_dev (arguments as for tgf_measure).
 * Limit: the array is 36 MiB (37748736 bytes) on every device that loads the library, held
 * until the process exits; a batch whose tgf_scratch_bytes exceeds it is rejected with
 * TGF_EINVAL and a message (about 41,000 sites in FP64, 82,000 in FP32 forms).
 * Set-up: the first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (that device must be current) and keeps it for the process; that first
 * call may also load the library's device code and commit the 36 MiB, so make it during set-up,
 * before any stream capture and outside latency-critical loops.  The kept address belongs to
 * the device's CUDA context: after cudaDeviceReset the call must not be used again.  No call of
 * tgf_measure_noalloc allocates or frees device memory.  All calls share the one array, which
 * keeps the last call's contents; each call overwrites everything it reads, so nothing needs
 * clearing, but calls whose kernels may overlap on the GPU (unordered streams) race. */
tgf_status tgf_measure_noalloc(int prec, const tgf_lattice *lat, int ncfg, const void *links,
                               tgf_obs *obs_dev, size_t obs_stride, int rec, double t,
                               unsigned flags, void *stream);

/* Time-slice topological charge q(x0, t) (Sec. 4): the clover charge density (eq. qlatt) summed
 * over the three directions other than `dir` at each slab x_dir = x, for every configuration at
 * the current field; q_dev[c * q_stride + x] for x = 0..L[dir]-1 (q_stride >= every L[dir]).
 * For the TGF box `dir` is a long direction (2 or 3), so the sum runs over both short ones.
 * FP64 sums in a fixed order; the slices of a configuration add up to its Q.  Uses the same
 * scratch as tgf_measure. */
tgf_status tgf_measure_slices(int prec, const tgf_lattice *lat, int ncfg, const void *links,
                              double *scratch, size_t scratch_bytes, int dir, double *q_dev,
                              size_t q_stride, unsigned flags, void *stream);

/* Flow every configuration c from t = 0 to t_end[c] (host array) in RK3 steps of eps: n_c =
 * floor(t_end[c]/eps) full steps, then one step of t_end[c] - n_c eps if that is > 1e-12 eps.
 * Observables are recorded into obs_dev[c * obs_cap + r] before every measure_every-th step
 * and once at t_end[c]; n_records[c] (host) receives the count.  `w` holds the start field and
 * receives the flowed one; `w_tmp` (same size) is the second ping-pong buffer; `accum` is X.
 * FP32 forms re-project onto SU(3) every `reunit_every` steps (0 = never).  By default the
 * whole flow is captured once into a CUDA graph and launched on `stream` (TGF_NO_GRAPH
 * launches the kernels directly).  Returns without synchronising. */
tgf_status tgf_flow(int prec, const tgf_lattice *lat, int ncfg, void *w, void *w_tmp, void *accum,
                    double *scratch, size_t scratch_bytes, double eps, const double *t_end,
                    int measure_every, int reunit_every, unsigned flags, tgf_obs *obs_dev,
                    size_t obs_cap, int *n_records, void *stream);

/* Number of records tgf_flow writes for one configuration (host arithmetic only). */
tgf_status tgf_flow_records(double eps, double t_end, int measure_every, int *n_records);

/* ---- library-owned context --------------------------------------------------------------- */

/* The stateful form of the calls above, for callers that want the library to own the device
 * memory: a context holds one batch (its lattices, precision, re-projection period and flags)
 * with its links, ping-pong buffer, accumulator, scratch, staging and records on one device.
 * Every call makes that device current and restores the caller's current device afterwards.
 * A context is not thread-safe; separate contexts are independent.
 *
 * tgf_create: validates as the stateless calls do and allocates everything (links zeroed);
 *   TGF_ENOMEM if cudaMalloc runs out of memory (nothing is left allocated), TGF_EINVAL for
 *   bad arguments or an unknown device.  flags: TGF_CLOVER_TRACELESS, TGF_NO_GRAPH.
 * tgf_destroy: frees everything (NULL is accepted).
 * tgf_set_links / tgf_get_links: configuration `cfg` from / to a host canonical buffer of
 *   exactly V * 72 doubles (synchronous).  tgf_set_links_device: from a device canonical buffer,
 *   enqueued on `stream`.
 * tgf_ctx_measure: {t, E, Q, P, S} of every configuration into out[ncfg] (host); synchronises
 *   `stream`; TGF_EKERNEL if a record is not finite.
 * tgf_ctx_flow: tgf_flow of the batch to t_end[c] (host array), records into out[c * cap + r]
 *   (host, cap >= tgf_flow_records of every configuration), counts into n_written[ncfg];
 *   synchronises `stream`; TGF_EKERNEL if a record is not finite.
 * tgf_ctx_save / tgf_ctx_load: tgf_save / tgf_load of the context's links. */
typedef struct tgf_ctx tgf_ctx;
tgf_status tgf_create(tgf_ctx **out, int device, int prec, int ncfg, const tgf_lattice *lat, int reunit_every,
                      unsigned flags);
void tgf_destroy(tgf_ctx *ctx);
tgf_status tgf_set_links(tgf_ctx *ctx, int cfg, const double *host_canon, size_t n_doubles);
tgf_status tgf_set_links_device(tgf_ctx *ctx, int cfg, const double *canon_dev, size_t n_doubles, void *stream);
tgf_status tgf_get_links(tgf_ctx *ctx, int cfg, double *host_canon, size_t n_doubles);
tgf_status tgf_ctx_measure(tgf_ctx *ctx, double t, tgf_obs *out, void *stream);
tgf_status tgf_ctx_flow(tgf_ctx *ctx, double eps, const double *t_end, int measure_every, tgf_obs *out, size_t cap,
                        int *n_written, void *stream);
tgf_status tgf_ctx_save(tgf_ctx *ctx, const char *path, double t, long long step, unsigned long long seed);
tgf_status tgf_ctx_load(tgf_ctx *ctx, const char *path, double *t, long long *step, unsigned long long *seed);

/* ---- SU(N) forms (FP64; Sec. 1, Sec. 3.1 with N colours, Sec. 5) ---------------------------- */

/* The paper defines the coupling for SU(N) on the l x l x (Nl) x (Nl) box with the twist
 * exp(2 pi i k / N) and gives numbers for N = 3; these calls run the same flow and measurement
 * for N = 2, 3, 4 in FP64: Z = -P_ta(U Sigma) with the 1/N trace, Luscher's RK3 as in tgf_stage,
 * exp(X) for N = 4 by a Taylor polynomial of degree 7 to 11 (chosen by ||X||_F, tail under
 * 1.1e-17) after scaling X by 2^-s to ||X||_F <= 1/5, evaluated by Paterson and Stockmeyer's
 * scheme, and squaring back (N = 2: the closed form e^{i tau}(cos theta + sin theta / theta X0);
 * N = 3: the Cayley-Hamilton form of tgf_stage), the
 * twisted clover and plaquette as in tgf_measure with the twist n_{mu nu} taken mod N and
 * P = (1/(6V)) sum_n sum_{mu<nu} (1/N) Re Tr[Z* P_{mu nu}].  Canonical buffers hold V x 4 x N x N
 * complex doubles per configuration ([x3][x2][x1][x0][mu][row][col][re,im]); device storage is
 * N^2 double2 planes per direction of Vp sites (Vp = V rounded up to 32), the accumulator N^2
 * reals per link.  Errors: TGF_EINVAL for N outside 2..4 and as for the SU(3) calls. */
tgf_status tgf_sun_links_bytes(int N, const tgf_lattice *lat, int ncfg, size_t *bytes);
tgf_status tgf_sun_accum_bytes(int N, const tgf_lattice *lat, int ncfg, size_t *bytes);
/* 4 doubles per 128-site block of every configuration, rounded up to 256 bytes */
tgf_status tgf_sun_scratch_bytes(int N, const tgf_lattice *lat, int ncfg, size_t *bytes);
tgf_status tgf_sun_pack(int N, const tgf_lattice *lat, int ncfg, const double *canon_dev, void *links, void *stream);
tgf_status tgf_sun_unpack(int N, const tgf_lattice *lat, int ncfg, const void *links, double *canon_dev,
                          void *stream);
/* One RK3 stage s = 1, 2, 3 of size eps for every link (the SU(N) counterpart of tgf_stage). */
tgf_status tgf_sun_stage(int N, const tgf_lattice *lat, int ncfg, const void *w_in, void *w_out, void *accum,
                         int stage, double eps, void *stream);
/* {t, E, Q, P, S} of every configuration into obs_dev[c * obs_stride + rec] (tgf_measure for SU(N);
 * flags: TGF_CLOVER_TRACELESS subtracts tr(G)/N). */
tgf_status tgf_sun_measure(int N, const tgf_lattice *lat, int ncfg, const void *links, double *scratch,
                           size_t scratch_bytes, tgf_obs *obs_dev, size_t obs_stride, int rec, double t,
                           unsigned flags, void *stream);

/* ---- ensemble generation (Sec. 3.1) ------------------------------------------------------ */

/* n_hybrid hybrid Monte Carlo sweeps of every configuration of `links` (TGF_FP64 storage), in
 * place: each is one heat-bath sweep followed by n_or over-relaxation sweeps, the algorithm the
 * paper uses to generate its ensembles (Sec. 3.1: one heat-bath sweep, then L~ over-relaxation
 * sweeps).  The action is the twisted Wilson action with beta = 18 b = 6/g0^2, so the weight of
 * a link U is exp((beta/3) Re Tr[U Sigma]), Sigma its twisted staple sum.  SU(3) is updated in
 * its three SU(2) subgroups (0,1), (0,2), (1,2) (Cabibbo-Marinari): heat-bath R = X v^+ with
 * X0 drawn by Kennedy-Pendleton (alpha > 2) or Creutz (otherwise), alpha = 2 beta k / 3;
 * over-relaxation R = (v^+)^2; U <- R U.  A sweep visits mu = 0..3, and for each the sites of
 * parity 0 then 1 (x0+x1+x2+x3 mod 2), so every extent must be even.
 * Random numbers are counter-based and reproducible: configuration c (index in this call) uses
 * key = h(seed, c), and draw `slot` of SU(2) subgroup g of link (site, mu) in heat-bath sweep
 * number w = first_sweep + h is h(key, (((w*4 + mu)*V + site)*3 + g)*260 + slot) with h(k, i) the
 * SplitMix64 output function of k + (i + 1) * 0x9E3779B97F4A7C15, mapped to
 * ((x >> 11) + 1) * 2^-53 in (0, 1]; slots 4a..4a+3 serve rejection attempt a < 64, slots 256
 * and 257 the direction of X; a subgroup with 64 rejected attempts is left unchanged.
 * Errors: TGF_EINVAL for another precision, an odd extent, beta <= 0 or not finite, negative
 * counts.  Enqueues 8 (1 + n_or) n_hybrid launches on `stream`. */
tgf_status tgf_mc_sweeps(int prec, const tgf_lattice *lat, int ncfg, void *links, double beta, int n_hybrid,
                         int n_or, unsigned long long seed, unsigned long long first_sweep, void *stream);

/* ---- self-checking builds ---------------------------------------------------------------- */

/* A library compiled with -DTGF_CHECK checks the site index of every link, accumulator and
 * clover access against the plane length in the kernels; a violation is recorded in a device
 * word of the kernel's source file and the access is redirected to site 0 (no fault).  This call
 * synchronises the device and returns the words as bits (1 stage kernels, 2 measurement, 4
 * layout, 8 Monte Carlo, 16 SU(N), 32 stage kernels of the other launch tiles) and clears them;
 * 0 means no violation since the last call.
 * In a normal build it returns TGF_EINVAL.  The paper has no counterpart: it replaces a memory
 * checker where none can run. */
tgf_status tgf_check_errors(unsigned int *bits);

/* ---- checkpoints --------------------------------------------------------------------------- */

/* Between RK3 steps the state of a flow is the field alone (X is rebuilt by stage 1), so a
 * checkpoint is the links in canonical FP64 with the flow time, the step count and a seed.
 * File (little-endian): 48-byte header {"TGFCKPT1", u32 version = 1, u32 ncfg, i32 precision the
 * links were stored in, i32 0, f64 t, i64 step, u64 seed}, then per configuration i32 L[4] and
 * i32 twist[6], then the canonical fields of all configurations (V x 72 doubles each), then the
 * CRC-32 (IEEE 802.3, as zlib's crc32) of everything before it.
 * tgf_save downloads `links` through the caller's staging buffer (as tgf_download; synchronises
 * `stream`) and writes `path`.  tgf_load reads and checks the whole file on the host first (magic,
 * version, CRC, size, and extents and twist mod 3 equal to `lat`), then uploads through the
 * staging buffer into `links` (any precision; FP32 forms round) and returns t, step and seed
 * (each pointer may be NULL).  Errors: TGF_EIO for a missing, unreadable, truncated or
 * corrupted file, TGF_EINVAL for a lattice mismatch or bad arguments; nothing is written to the
 * device unless the file passes every check. */
tgf_status tgf_save(const char *path, int prec, const tgf_lattice *lat, int ncfg, const void *links, double *staging_dev,
                    size_t staging_bytes, double t, long long step, unsigned long long seed, void *stream);
tgf_status tgf_load(const char *path, int prec, const tgf_lattice *lat, int ncfg, void *links, double *staging_dev,
                    size_t staging_bytes, double *t, long long *step, unsigned long long *seed, void *stream);
/* CRC-32 of n bytes (the checkpoint checksum; host only). */
unsigned int tgf_crc32(const void *data, size_t n);

/* ---- coupling (host only) ----------------------------------------------------------------- */

/* N(c, Lt) of eq. (latt_norm) for SU(N): the inverse of
 * (c^4/128) sum_{mu!=nu} sum'_q exp(-c^2 Lt^2 qhat^2/4) sin^2(q_nu) cos^2(q_mu/2)/qhat^2
 * over q_mu = 2 pi n_mu/Lt, n_mu = 0..Lt-1, dropping n_0 = n_1 = 0 (mod N).  O(Lt^4) work. */
tgf_status tgf_norm(double c, int Ltilde, int N, double *norm_out);

/* lambda_TGF = N(c, Lt) t^2 sum_i E_i d_i / (3 sum_i d_i), d_i = [|Q_i| < 1/2] (eq. lambdat_latt).
 * Returns TGF_ESTATE (and n_kept = 0) when no configuration passes the cut. */
tgf_status tgf_lambda(double c, int Ltilde, double t, const double *E, const double *Q, int ncfg,
                      double *lambda_out, int *n_kept);

/* Correlator of the time-slice charge in the zero-charge sector (eq. qcorr), host only:
 * C[d] = sum_c delta_c (1/T) sum_x q_c(x + d) q_c(x) / sum_c delta_c, d = 0..T-1 (periodic),
 * delta_c = [|Q_c| < 1/2]; q is [ncfg][q_stride] (T <= q_stride).  TGF_ESTATE when no
 * configuration is kept. */
tgf_status tgf_slice_correlator(const double *q, size_t q_stride, const double *Q, int ncfg, int T,
                                double *C_out, int *n_kept);

/* ---- diagnostics ---------------------------------------------------------------------------- */

/* FMA-pipe peak of the current device in TFLOP/s (2 flops per FMA) for TGF_FP64 or TGF_FP32:
 * the roofline denominator of the flow kernels, which are bound by vector FP arithmetic.  With
 * TGF_FMA_PEAK_FP32X2 the same chains run as packed fma.rn.f32x2 pairs, with
 * TGF_FMA_PEAK_FP32_MIXED as packed and scalar FMAs interleaved: the FP32 flow kernels use
 * packed pairs, so these check that no mix of the two forms exceeds the scalar FP32 peak.  The
 * paper has no counterpart; this is a measurement aid.  `sink_dev` is a caller-owned device
 * buffer of at least blocks_per_sm * (number of SMs) * 8 bytes that the kernel may write;
 * the call synchronises `stream`. */
#define TGF_FMA_PEAK_FP32X2 3
#define TGF_FMA_PEAK_FP32_MIXED 4
tgf_status tgf_fma_peak(int prec, void *sink_dev, int blocks_per_sm, int iters, double *tflops,
                        void *stream);

const char *tgf_last_error(void);
const char *tgf_status_string(int status);
/* Library version, "major.minor.patch". */
const char *tgf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TGF_H */
