/*
 * art.h -- C ABI of the GB300 adaptive ray tracing (ART) library.
 *
 * The library traces the direct radiation of point sources through a uniform 3-D
 * Cartesian grid with adaptive HEALPix rays, as in Kim, Kim, Ostriker & Skinner (2017),
 * Sec. 2.1: photon packets leave each source along the 12*4^l0 nested HEALPix directions
 * with L/N_ray each; each packet is walked cell by cell and loses
 * dL = L (1 - exp(-chi ds)) in every cell it crosses (Eq. e:RT2), with
 * chi = n_H0 sigma_H + n_H sigma_d (Sec. 2.3); the cell accumulates sum dL/chi and
 * sum dL n (Eqs. e:Erad, e:Frad); a ray splits into its four children at level l+1 when it
 * reaches r_max(l) = [3/(pi m_ray)]^(1/2) 2^l dx; it is retired when it leaves the grid or
 * when its optical depth from the source exceeds tau_max.
 *
 * Units: code units with c = 1 and h nu_i = 1. Luminosities are photon rates, so
 *   gamma[c]  = sigma_H / dV * sum dL/chi          (Eq. e:photrate2 divided by n_HI)
 *   energy[c] = 1 / dV * sum dL/chi                 (Eq. e:Erad)
 *   force[a][c] = 1 / dV * sum dL n_a               (chi F / c with Eq. e:Frad)
 * Cells are indexed i + nx*(j + ny*k) (x fastest), i.e. a C array [nz][ny][nx].
 *
 * Conventions for every entry point:
 *   - the return value is ART_OK (0) or a negative ART_E* status; nothing aborts, throws or
 *     exits across the ABI; art_strerror names a status;
 *   - "device" pointers are CUDA device memory on the grid's device, borrowed from the
 *     caller, never freed by the library; "host" pointers are ordinary host memory, read
 *     or written only during the call;
 *   - work is enqueued on the CUDA stream given to art_create_grid, in call order; a call
 *     returns before the GPU work finishes unless it says it synchronizes;
 *   - a grid object is not thread-safe: one host thread at a time per grid.
 */
#ifndef ART_H
#define ART_H

#ifdef __cplusplus
extern "C" {
#endif

#define ART_OK 0
#define ART_EINVAL (-1)          /* bad argument, size or input value */
#define ART_ENOMEM (-2)          /* device or pinned host allocation failed */
#define ART_EQUEUE_OVERFLOW (-3) /* a ray front exceeded its capacity; results incomplete */
#define ART_ETIMEOUT (-4)        /* a bounded device wait ran out; results incomplete */
#define ART_EACCOUNTING (-5)     /* retired-ray weights do not add up to N_src*12*4^l_max */
#define ART_ECUDA (-6)           /* a CUDA runtime call failed */
#define ART_ESTATE (-7)          /* call out of order (e.g. no sources, no trace yet) */
#define ART_EINTERNAL (-8)       /* a device-side consistency bound was exceeded (a walk
                                    longer than any straight ray through the grid, a schedule
                                    phase without rays); results incomplete */

#define ART_MAX_LEVEL 13
#define ART_NLEVELS 20

/* Schedules of art_trace. */
#define ART_SCHED_PERSISTENT 0 /* all sources in one cooperative launch, device work queue */
#define ART_SCHED_PLAIN 1      /* one source at a time, one launch per HEALPix level */

/* Flags of art_params.flags */
#define ART_F_ROTATE 1u        /* apply art_params.rot to every HEALPix direction */

typedef struct art_grid art_grid; /* opaque, owned by the library */

/* Trace parameters (Sec. 2.1, Sec. 2.3). Fill with art_params_default, then override. */
typedef struct {
    int level0;          /* base HEALPix level l0, 0..12 (paper default 4) */
    int level_max;       /* < 0: per source, the smallest l >= l0 whose r_max reaches the
                            farthest box corner, capped at 13; else a fixed l_max, l0..13 */
    double m_ray;        /* split criterion: rays per cell face (paper default 4) */
    double tau_max;      /* retire a ray once tau > tau_max (paper default 7) */
    double sigma_H;      /* H photoionization cross section (code units) */
    double sigma_d;      /* dust cross section per H; used only with a total-density field */
    double rot[9];       /* row-major rotation of the ray directions (with ART_F_ROTATE) */
    unsigned flags;      /* ART_F_* */
    int schedule;        /* ART_SCHED_* */
    int block_threads;   /* threads per block of the trace kernels (0 = library choice) */
    int chunk;           /* rays a warp takes from the queue at a time (0 = library choice) */
    long long queue_capacity; /* rays per level buffer beyond l0 (0 = library choice) */
    double wait_limit_s; /* bound on any device-side wait (grid barrier); 0 = library default
                            (60 s); a negative value makes every wait give up at once. A
                            block waits at a barrier while the slowest block finishes its
                            share of one phase of the schedule, so grids and source sets
                            whose phases run longer than the bound need a larger value
                            (the trace then fails with ART_ETIMEOUT, results incomplete) */
    int blocks_per_sm;   /* resident blocks per SM of the persistent trace (0 = as many as
                            fit); fewer blocks keep fewer rays in flight */
    double d_max;        /* > 0: every ray ends at this distance from its source (the cutoff
                            of the weak-scaling test, Sec. 3.1), its remaining L counted as
                            escaped; at d_max = r_max(l) the cut wins over the split.
                            <= 0: no cutoff (default). NaN or inf: ART_EINVAL */
} art_params;

/* Counters of one trace (tallies in FP64). */
typedef struct {
    unsigned long long crossings;                 /* emitted cell segments of length > 0 */
    unsigned long long rays_total;                /* rays traced, all levels */
    unsigned long long rays_per_level[ART_NLEVELS];
    unsigned long long destroy;                   /* sum of 4^(l_max - l) over retired rays */
    unsigned long long destroy_expected;          /* N_src * 12 * 4^l_max */
    double L_in, L_absorbed, L_escaped, L_dropped; /* photon bookkeeping */
    int level_reached;
    int level_max;                                /* l_max over all sources */
    int status;                                   /* device-side status of the trace */
    int pad;
    /* the non-ionizing bin of a two-bin trace (zero otherwise) */
    double Ln_in, Ln_absorbed, Ln_escaped, Ln_dropped;
} art_stats;

/* Fills p with the paper's defaults: l0 = 4, m_ray = 4, tau_max = 7, sigma_H = 1,
 * sigma_d = 0, identity rotation, persistent schedule, library-chosen launch knobs. */
void art_params_default(art_params* p);

/* Creates a grid of nx*ny*nz cells of side dx whose lower corner is box_lo[3]: the uniform
 * Cartesian grid through which rays are traced (Sec. 2.1), holding the neutral and total
 * hydrogen densities from which the opacity chi_i = n_HI sigma_H + n_H sigma_d is formed
 * (Sec. 2.3).
 * d_nH0: device, nx*ny*nz floats, neutral H density (required, finite, >= 0).
 * d_nH: device, total H density for the dust term, or NULL for no dust.
 * stream: a cudaStream_t (NULL = legacy default stream) on the current device; all work of
 * this grid is ordered on it. The field pointers are borrowed and must stay valid until the
 * next art_update_fields or art_destroy_grid. Allocates the per-cell accumulators
 * (16 B per cell) and scratch. Errors: ART_EINVAL (sizes <= 0, more than 2^31 cells, dx <= 0,
 * d_nH0 NULL), ART_ENOMEM, ART_ECUDA. */
int art_create_grid(art_grid** out, int nx, int ny, int nz, const double box_lo[3], double dx,
                    const float* d_nH0, const float* d_nH, void* stream);

/* Re-points the density fields (same sizes and ownership rules as at creation): the n_HI
 * (and n_H) of Sec. 2.3, which change between radiation substeps as the neutral fraction is
 * updated (Eq. e:xn3, then n_HI = x_n n_H). The fields are read again by every trace, so
 * updating their contents in place needs no call. Errors: ART_EINVAL (g or d_nH0 NULL). */
int art_update_fields(art_grid* g, const float* d_nH0, const float* d_nH);

/* Appends n point sources at x_src with luminosity L (Sec. 2.1: each injects L/N_ray(l0)
 * along every base-level HEALPix direction; several sources add their rays' deposits).
 * h_pos: host, n*3 doubles (x, y, z), each strictly inside the box.
 * h_L: host, n doubles, luminosities >= 0 (photon rates). The arrays are copied.
 * Errors: ART_EINVAL (n < 0, a source on or outside the box boundary, negative or
 * non-finite luminosity). */
int art_add_sources(art_grid* g, int n, const double* h_pos, const double* h_L);

/* Gives every source currently held a second, non-ionizing luminosity (Sec. 2.3): the trace
 * then carries two frequency bins on each ray -- the ionizing one, attenuated by
 * chi_i = n_H0 sigma_H + n_H sigma_d, and a non-ionizing one attenuated by dust alone,
 * chi_n = n_H sigma_d (requires the total-density field d_nH for any attenuation) -- and the
 * force output sums the momentum of both (Eq. e:radforce); gamma and energy stay those of
 * the ionizing bin. A packet is retired once its dust-only optical depth (never larger than
 * the ionizing one) exceeds tau_max. h_Ln: host, art_num_sources doubles >= 0, copied;
 * sources added later get 0. NULL switches the second bin off. art_trace_backward covers
 * one-bin traces only (ART_EINVAL with a second bin). Errors: ART_EINVAL, ART_ESTATE. */
int art_set_nonionizing(art_grid* g, const double* h_Ln);

/* Removes all sources (and their non-ionizing luminosities). */
int art_clear_sources(art_grid* g);

/* Number of sources currently held. */
int art_num_sources(const art_grid* g);

/* One full trace of all sources (Sec. 2.1), overwriting the outputs:
 *   d_gamma:  device, ncell floats: photoionization rate per neutral atom (required);
 *   d_force:  device, 3*ncell floats, SoA blocks x, y, z: radiation force density, or NULL;
 *   d_energy: device, ncell floats: radiation energy density, or NULL.
 * h_stats: host, or NULL. With h_stats the call synchronizes the stream, fills the counters
 * and returns the trace's device status (ART_EQUEUE_OVERFLOW, ART_ETIMEOUT, ART_EACCOUNTING);
 * without it the call only enqueues work and art_get_stats reports later. The first call
 * for a given (l_max, level0, sources) allocates ray buffers and direction tables, so do one
 * untimed call before capturing a stream into a CUDA graph.
 * Errors: ART_EINVAL (bad parameters: level0 outside 0..12, level_max outside l0..13,
 * m_ray <= 0, tau_max <= 0, sigma < 0, chunk not a multiple of 32, block_threads not a
 * multiple of 32 in 64..1024, queue_capacity < 4), ART_ESTATE (no sources), ART_ENOMEM,
 * ART_ECUDA. */
int art_trace(art_grid* g, const art_params* p, float* d_gamma, float* d_force,
              float* d_energy, art_stats* h_stats);

/* Synchronizes the grid's stream and copies the counters of the last trace (or backward
 * trace). Returns the device status of that trace. ART_ESTATE if nothing was traced. */
int art_get_stats(art_grid* g, art_stats* h_stats);

/* Gradient of loss = sum_c (w_c gamma_c + v_c . force_c) for the current fields and sources
 * (new; the paper has no adjoint; the forward map is the trace of Sec. 2.1 with the opacity
 * of Sec. 2.3): recomputes every ray's path in reverse level order instead of storing
 * segments, summing child-ray adjoints into their parents.
 *   d_w:          device, ncell floats, dloss/dgamma per cell, or NULL (no gamma term);
 *   d_v:          device, 3*ncell floats (SoA blocks x, y, z, like art_trace's d_force),
 *                 dloss/dforce per cell, or NULL (no force term); not both NULL;
 *   d_dlog_nH0:   device, ncell floats, output dloss/dlog(n_H0) per cell (overwritten);
 *   d_dL:         device, n_src doubles, output dloss/dL per source (overwritten), or NULL.
 *                 Device memory (not host) so that the call never synchronizes and can sit
 *                 in a CUDA graph or in a torch autograd backward without a host round trip;
 *                 callers copy the n_src doubles out when they need them.
 * Split points and tau_max retirement are held fixed. A force term doubles the per-step
 * gather (32-byte cell records, 32 B x ncell of library memory). One-bin traces only
 * (ART_EINVAL with a second bin). Same parameters and status rules as art_trace; h_stats
 * as in art_trace, with crossings, rays per level and the destroy counter; its photon
 * tallies (escaped, dropped) are zero, because the reverse sweep walks rays of unit
 * source luminosity. */
int art_trace_backward(art_grid* g, const art_params* p, const float* d_w, const float* d_v,
                       float* d_dlog_nH0, double* d_dL, art_stats* h_stats);

/* Neutral-fraction update of every cell over dt (Sec. 2.3), elementwise on the stream:
 *   method 0: Eq. e:xn3 (electron density held at n_H (1 - x_n) over the step);
 *   method 1: Eq. e:xn2 (exact quadratic solution), with the Gamma = 0 solution where
 *             gamma is 0.
 * d_gamma (ncell floats, photoionization rate), d_nH (ncell floats, total H density) are
 * read; d_xn (ncell floats, neutral fraction in [0,1]) is updated in place; d_nH0, if not
 * NULL, receives x_n n_H (the neutral density for the next trace). alpha_B > 0, dt >= 0.
 * Errors: ART_EINVAL, ART_ECUDA. */
int art_xn_update(void* stream, long long ncell, const float* d_gamma, const float* d_nH,
                  float* d_xn, float* d_nH0, double alpha_B, double dt, int method);

/* Substep size of Eq. e:dtss: C * min over cells of n_H / |I - R|, with
 * I = x_n n_H gamma and R = alpha_B (n_H (1 - x_n))^2, written to d_dt (device, 1 double;
 * +inf when I = R everywhere). d_scratch: device, at least art_dt_scratch_bytes(ncell)
 * bytes. Errors: ART_EINVAL, ART_ECUDA. */
int art_dt_substep(void* stream, long long ncell, const float* d_gamma, const float* d_nH,
                   const float* d_xn, double alpha_B, double C, void* d_scratch, double* d_dt);
long long art_dt_scratch_bytes(long long ncell);

/* Largest ncell accepted by art_dt_substep_static. */
#define ART_DT_STATIC_MAX_CELLS (1ll << 24)

/* The substep size of art_dt_substep, for callers that cannot allocate device memory (the
 * paper has no counterpart): the same result, with the per-block partial minima held in a
 * fixed array inside the library (256 KB, one float per 256-cell tile) instead of caller
 * scratch. Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * d_gamma, d_nH, d_xn: device, ncell floats each (read); d_dt: device, 1 double (written).
 * Limits and sharing:
 *   - ncell must be in 1..ART_DT_STATIC_MAX_CELLS (2^24); larger inputs return ART_EINVAL
 *     with nothing enqueued;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the life of the
 *     process; make that first call before any stream capture. The kept address belongs to
 *     the device's primary context: after cudaDeviceReset on a device this entry point must
 *     not be called on that device again;
 *   - every call on a device shares the one array, which keeps the last call's partials;
 *     each call writes every partial it reads, so no clearing is needed, but calls whose
 *     GPU work overlaps (different streams, no ordering between them) race and give wrong
 *     results: order them on one stream or with events.
 * Errors: ART_EINVAL, ART_ECUDA. */
int art_dt_substep_static(void* stream, long long ncell, const float* d_gamma,
                          const float* d_nH, const float* d_xn, double alpha_B, double C,
                          double* d_dt);

/* Splitting one trace over several GPUs by source (new; the paper's MPI version decomposes the
 * domain and passes rays between ranks instead, Sec. 2.2). Sources are independent and
 * their deposits add (Sec. 2.1), so ranks holding the same density field can each trace a
 * disjoint subset of the sources and sum gamma, force and energy with one all-reduce; the
 * reverse sweep's dloss/dlog n_H0 sums the same way, dloss/dL_s belongs to the source's rank.
 *
 * art_estimate_work: a per-source estimate of the trace's crossings, for balancing that
 * split. Walks 12*4^min(l0, 2) rays from every source, without splitting, to where the trace
 * would retire them (tau > tau_max with the current fields and p's cross sections, the d_max
 * cutoff, or the grid boundary); a coarse ray reaching D cells covers the base rays out to
 * r_max(l0) and about m_ray Omega r^2 split rays at radius r beyond it.
 * h_work: host, art_num_sources doubles (written), in crossings (an estimate, not a count).
 * Synchronizes the grid's stream; allocates and frees a small scratch.
 * Errors: ART_EINVAL, ART_ESTATE (no sources), ART_ENOMEM, ART_ECUDA. */
int art_estimate_work(art_grid* g, const art_params* p, double* h_work);

/* Assigns n sources with work estimates h_work (host, n doubles >= 0) to nranks ranks:
 * longest processing time first (largest estimate first, each to the least-loaded rank,
 * ties by index), so every rank computes the same assignment from the same estimates and the
 * largest load is at most 4/3 of the optimum. h_rank: host, n ints (written, 0..nranks-1);
 * h_load: host, nranks doubles (written, the summed estimate per rank), or NULL.
 * Host only: needs no GPU. Errors: ART_EINVAL (n < 0, nranks < 1, negative or non-finite
 * work, NULL arrays). */
int art_partition_sources(int n, const double* h_work, int nranks, int* h_rank, double* h_load);

/* Frees the grid and everything it allocated (not the borrowed fields). NULL is a no-op. */
void art_destroy_grid(art_grid* g);

/* Static description of a status code. */
const char* art_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* ART_H */
