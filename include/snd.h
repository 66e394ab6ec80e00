/*
 * snd.h - C ABI of the GB300 Spiking Neural Dedispersion (SND) hot path.
 *
 * The library searches a streamed uint8 filterbank for dispersed pulses:
 *   delta encoder  -> SND delay-and-add tree -> DM-scaled boxcar matched filter
 *   -> threshold, 9x9 closing, 8-connected labelling -> candidate list
 * (arXiv 2606.15361, Methods: "Pipeline overview", "Input encoding", "The Spiking
 * Neural Dedispersion algorithm", "Matched filtering", "Candidate detection").
 *
 * Conventions shared by every entry point:
 *  - Return value: SND_OK (0) on success, a negative snd_status_t otherwise. No C++
 *    exception crosses this boundary. An error raised while a plan is executing is
 *    sticky: later calls on that plan return it until snd_destroy.
 *  - "device" pointers are CUDA global-memory pointers of the current device; "host"
 *    pointers are ordinary CPU memory (pinned memory makes snd_execute_host faster).
 *  - stream is a cudaStream_t passed as void* (0 = the legacy default stream).
 *  - A plan is not re-entrant: one stream at a time per plan. Distinct plans may run
 *    concurrently on distinct streams and workspaces.
 *  - The library allocates no device memory. All device state lives in a
 *    caller-owned workspace (snd_workspace_size / snd_bind_workspace).
 */
#ifndef SND_H
#define SND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SND_OK = 0,
  SND_ERR_ARG = -1,          /* invalid argument (null pointer, size, option range) */
  SND_ERR_FREQ_ORDER = -2,   /* channel frequencies not finite, positive, distinct */
  SND_ERR_DM = -3,           /* a trial DM is negative or not finite */
  SND_ERR_WORKSPACE = -4,    /* workspace missing, too small or misaligned */
  SND_ERR_CHUNK = -5,        /* nsamp <= 0 or > max_chunk */
  SND_ERR_CUDA = -6,         /* a CUDA runtime call failed */
  SND_ERR_STATE = -7,        /* call not valid in the plan's current state */
  SND_ERR_TIMEOUT = -8,      /* a bounded device-side loop gave up */
  SND_ERR_OVERFLOW = -9,     /* a fixed-capacity device list overflowed (results dropped) */
  SND_ERR_NOMEM = -10,       /* host allocation failed */
  SND_ERR_UNSUPPORTED = -11  /* configuration outside what the GPU kernels implement */
} snd_status_t;

/* Tree activation modes (Methods, "Tree activation modes"). */
typedef enum {
  SND_MODE_BINARY = 0,  /* Mode A: node = 1[count >= K] (K_L at leaves, K_I above) */
  SND_MODE_GRADED = 1,  /* Mode B: node = min(sum, N) at every node, root included */
  SND_MODE_FLOAT = 2,   /* Mode C: node = sum; root divided by sqrt(N_f) */
  /* Mode C with the labelled payload x_c(t) = z_c(t) * 1[P_c(t) >= u_c], z = (P - mu_c)/sigma_c
     (the encoder's clipped per-chunk statistics), for the float-mode precision study: every
     node below the root is stored in FP32, or FP16 with SND_FLAG_FP16_PARTIALS, before its
     parent adds it in FP32, children in index order; the FP32 root times fp32(1/sqrt(N_f)) is
     the plane. Produces the float32 plane only: the matched filter and candidate stages do not
     run (snd_candidates returns none). */
  SND_MODE_ZFLOAT = 3
} snd_mode_t;

typedef struct snd_plan_s* snd_plan_t;

/* Option flag: evaluate the tree with the slow scalar verification kernel (one thread per
 * DM-sample, integer counts from the full delay table) instead of the tiled bit-sliced
 * kernel, and the mask closing as four separate separable passes instead of the fused
 * tiled kernel. Results are identical; it exists to cross-check the fast kernels. */
#define SND_FLAG_REFERENCE_TREE 1
/* Option flag (SND_MODE_ZFLOAT only): store the payload and every partial sum below the root
 * in FP16 (round to nearest even) instead of FP32; accumulation stays FP32. */
#define SND_FLAG_FP16_PARTIALS 2
/* Option flag: evaluate the tree with the leaf-sharing kernel (distinct leaf patterns of a DM
 * tile evaluated once, then gathered per DM) even where the direct kernel applies. Results
 * are identical; it keeps the paper's shared-leaf evaluation available for comparison. */
#define SND_FLAG_LEAF_SHARING 4
/* Option flag (SND_MODE_ZFLOAT only): the payload of a spike is 1 (the paper's own 0/1 raster)
 * instead of z, so every node holds a spike count and the storage type alone decides the
 * plane's error (FP16 holds every count up to 2048 exactly). */
#define SND_FLAG_UNIT_PAYLOAD 16
/* Option flag (binary, graded, float): count, per tree level, the node-samples whose output is
 * nonzero over the emitted samples (the per-level fire rates of Supplementary Table S2 that the
 * paper's dynamic-power model uses); read them with snd_level_rates. Needs the direct tree
 * kernel with C = 4 (nchan a multiple of 64, at most 13 levels); otherwise the plan returns
 * SND_ERR_UNSUPPORTED. Float and graded plans pay one extra counting pass per chunk. */
#define SND_FLAG_LEVEL_RATES 32

/*
 * Options. Fill with snd_options_init(mode, &o) (Supplementary Table S1 operating point
 * for that mode) and then override fields; values are used as given.
 */
typedef struct {
  int32_t cluster_size;     /* C, leaf cluster size, 1..7 (Table S1: 4) */
  int32_t k_leaf;           /* K_L, binary leaf quorum, 1..8 (Table S1: 2); other modes ignore */
  int32_t k_internal;       /* K_I, binary internal quorum, 1..8 (Table S1: 2) */
  int32_t graded_cap;       /* N, graded cap, 1..255 (Table S1: 255) */
  double enc_theta;         /* theta, encoder threshold in sigma (1.5 binary/float, 0.75 graded) */
  double det_theta;         /* Theta, detection S/N threshold, > 0 (Table S1: 7.0) */
  double sigma_min;         /* sigma floor of the matched filter, binary mode only (0.20) */
  double mf_alpha;          /* alpha of the width rule (Methods, "Matched filtering": 0.1) */
  int32_t closing_size;     /* closing element side, odd, 1..31 (9) */
  int32_t n_min_pixels;     /* islands with fewer closed-mask pixels are dropped (10) */
  int32_t max_chunk;        /* largest nsamp accepted by snd_execute (default 32768) */
  int32_t cand_capacity;    /* candidates held on the device between snd_candidates calls */
  int32_t cell_capacity;    /* mask cells with S/N kept per matched-filter block */
  int32_t run_capacity;     /* closed-mask runs per matched-filter block */
  int32_t flags;            /* 0 or SND_FLAG_REFERENCE_TREE / SND_FLAG_LEAF_SHARING / SND_FLAG_LEVEL_RATES,
                               or SND_FLAG_FP16_PARTIALS / SND_FLAG_UNIT_PAYLOAD (zfloat) */
  int32_t plane_dtype;      /* d_plane_out element type: 0 = int32 / float32 (default); 1 = uint8,
                               binary and graded modes only (their roots are 0..255) */
  int32_t tree_warps;       /* direct tree kernel: warps per CTA, 2, 4 or 8 (0 = 8); a CTA covers
                               32 trial DMs x warps x (2 or 4) output words. Results never depend on it */
  int32_t tree_round;       /* direct tree kernel: channels staged per round, 64 or 128 (0 = 128 where
                               it fits two CTAs per SM, else 64). Results never depend on it */
} snd_options_t;

/* One detection (Methods, "Candidate detection": one candidate per island, peak pixel). */
typedef struct {
  int32_t dm_index;   /* row of the trial-DM grid */
  float dm;           /* dm_grid[dm_index] */
  int64_t t;          /* stream sample index (time of arrival at the top of the band) */
  float snr;          /* peak S/N (FP64 matched filter, rounded to float) */
  int32_t width;      /* boxcar width of the peak, samples */
  int32_t npix;       /* pixels of the island in the closed mask */
  int32_t reserved;
} snd_candidate_t;

typedef struct {
  int32_t nchan, ndm, mode, branching, cluster_size;
  int32_t max_delay;               /* D = max delta_c(d), samples */
  int32_t nlevels;                 /* tree levels including the leaves */
  int32_t nodes_per_level[24];     /* structural nodes per level (leaves first) */
  int64_t unique_per_level[24];    /* distinct node patterns per level (neuron count) */
  double adds_per_dm_sample;       /* additions per DM-sample with pattern sharing */
  int32_t wmax;                    /* largest boxcar width over the DM grid */
  int32_t ring_words;              /* bit-ring words per channel (one copy) */
  int64_t hist_mem_bytes;          /* Eq. hist_mem for this single band and mode */
  size_t workspace_bytes;
  int64_t samples_in;              /* samples consumed so far */
  int64_t emitted;                 /* E: plane samples emitted per row so far */
  int64_t scored;                  /* F: start times scored by the matched filter so far */
  int32_t candidates_pending;      /* -1 unless synchronised by snd_candidates */
  int32_t tree_tile_dms;           /* DM rows per tree CTA */
  int32_t tree_tile_words;         /* 32-sample words per tree CTA */
  int32_t tree_group_leaves;       /* leaves staged per shared-memory round */
  int32_t tree_smem_bytes;         /* dynamic shared memory of the tree kernel */
  int32_t max_patterns_per_group;
  int64_t kernel_launches;         /* CUDA kernels enqueued by this plan since binding */
  int32_t tree_kernel;             /* 0 leaf-sharing k_tree, 1 direct k_snd, 2 reference, 3 labelled payload */
  int32_t device_status;           /* device status bits read by the last snd_candidates (0 = clean):
                                      1 matched-filter cells, 2 runs, 4 candidates, 8 block candidates
                                      overflowed; 16 threshold search, 32 union-find, 128 tree staging
                                      wait, 256 grid barrier wait, 512 matched-filter staging wait
                                      gave up; 64 a cell outside its run */
} snd_plan_stats_t;

/* Pipeline stages timed by snd_profile / snd_profile_read. */
enum { SND_STAGE_ENCODE = 0, SND_STAGE_TREE = 1, SND_STAGE_MF = 2, SND_STAGE_CANDIDATES = 3, SND_NUM_STAGES = 4 };

/* Fill *o with the Supplementary Table S1 operating point of `mode`. */
int snd_options_init(snd_mode_t mode, snd_options_t* o);

/*
 * Build a plan (host only; no CUDA call).
 *   freqs_mhz[nchan]  channel-centre frequencies, MHz, any order, distinct, > 0
 *   dt_s              sample interval, seconds, > 0
 *   dm_grid[ndm]      trial DMs, pc cm^-3, finite and >= 0, any order, duplicates allowed
 *   branching         B >= 2 (Methods, "Tree levels")
 * Delays: delta_c(d) = floor(K d (f_c^-2 - f_ref^-2)/dt + 1/2), K = 4.148808e3 MHz^2 s,
 * f_ref = highest frequency (Methods, "Incoherent dedispersion").
 * snd_plan uses the Table S1 options of `mode`. *out receives the plan (NULL on error).
 */
int snd_plan(const double* freqs_mhz, int32_t nchan, double dt_s, const double* dm_grid,
             int32_t ndm, int32_t branching, snd_mode_t mode, snd_plan_t* out);
int snd_plan_ex(const double* freqs_mhz, int32_t nchan, double dt_s, const double* dm_grid,
                int32_t ndm, int32_t branching, snd_mode_t mode, const snd_options_t* opts,
                snd_plan_t* out);

/* Bytes of device workspace the plan needs (0 for a NULL plan). */
size_t snd_workspace_size(snd_plan_t plan);

/*
 * Bind a device workspace of at least snd_workspace_size bytes, 256-byte aligned, and reset
 * the stream state (stream time back to 0). The caller owns the memory and must keep it
 * alive until snd_destroy or the next bind. Uploads the plan's device tables and clears the
 * workspace with work enqueued on `stream` (no host synchronisation).
 */
int snd_bind_workspace(snd_plan_t plan, void* d_workspace, size_t bytes, void* stream);

/*
 * Process the next chunk of the stream (Methods, "Pipeline overview").
 *   d_chunk      device uint8[nsamp][nchan] (time-major, SIGPROC order), read only;
 *                must stay valid until the stream passes this call
 *   nsamp        1..max_chunk samples
 *   stream       all work is enqueued on it; no host synchronisation
 *   d_plane_out  optional device output [ndm][*nemit_out] row-major: int32 root values
 *                (binary 0/1, graded 0..N; uint8 with plane_dtype = 1) or float32 (float mode, counts/sqrt(N_f); zfloat,
 *                the labelled-payload plane) for the newly emitted samples [E_prev, E_new);
 *                NULL to skip
 *   nemit_out    optional host int32: E_new - E_prev, the emitted samples per row, where
 *                E = max(0, samples consumed - D) (every emitted sample has full history)
 * Candidates found by this call accumulate on the device until snd_candidates.
 */
int snd_execute(snd_plan_t plan, const uint8_t* d_chunk, int32_t nsamp, void* stream,
                void* d_plane_out, int32_t* nemit_out);

/*
 * Same as snd_execute for a HOST chunk: copies h_chunk into one of the workspace's two
 * staging areas and then runs the path on `stream`. The copy runs on a private stream of
 * the plan that waits only for the chunk before last (the previous user of that staging
 * area), so it overlaps the previous chunk's kernels; the work on `stream` waits for the
 * copy. h_chunk must therefore already hold the chunk when the call is made (it may be read
 * before earlier work on `stream` completes) and stay unchanged until `stream` passes this
 * chunk; page-locked memory makes the copy asynchronous.
 */
int snd_execute_host(snd_plan_t plan, const uint8_t* h_chunk, int32_t nsamp, void* stream,
                     void* d_plane_out, int32_t* nemit_out);

/*
 * Synchronise the plan's last stream, copy the candidates accumulated since the previous
 * call to host_out (at most cap; sorted by (t, dm_index)), report their count in *n_out
 * and clear the device list. Returns SND_ERR_OVERFLOW (after copying what was kept) when
 * a device capacity overflowed since the last call, SND_ERR_TIMEOUT when a bounded device
 * loop gave up.
 */
int snd_candidates(snd_plan_t plan, snd_candidate_t* host_out, int32_t cap, int32_t* n_out);

/* Plan statistics (host only; stream counters are those of the last enqueued call). */
int snd_plan_stats(snd_plan_t plan, snd_plan_stats_t* out);

/*
 * Per-level fire counts of a plan made with SND_FLAG_LEVEL_RATES (Supplementary Table S2):
 * fires_out[l] (nullable) = node-samples of tree level l (0 = leaves) with a nonzero output,
 * rates_out[l] (nullable) = fires / (nodes of level l x ndm x samples emitted per row), both
 * accumulated since the workspace was bound; for l < min(cap, nlevels). *nlevels_out = levels.
 * Synchronises the plan's last stream. SND_ERR_STATE without the flag or before binding.
 */
int snd_level_rates(snd_plan_t plan, uint64_t* fires_out, double* rates_out, int32_t cap, int32_t* nlevels_out);

/* Copy the plan's integer delay table int32[ndm][nchan] to host memory (n >= ndm*nchan). */
int snd_delay_table(snd_plan_t plan, int32_t* host_out, int64_t n);

/*
 * Per-stage device timing. enable != 0 makes every following snd_execute record a CUDA
 * event pair around each stage on the execution stream (events are created on first use
 * and kept by the plan); enable == 0 stops recording. snd_profile_read synchronises the
 * recorded events, writes the summed milliseconds and the number of timed launches of each
 * stage into ms_out[SND_NUM_STAGES] and count_out[SND_NUM_STAGES] (either may be NULL), and
 * clears the record.
 */
int snd_profile(snd_plan_t plan, int enable);
int snd_profile_read(snd_plan_t plan, double* ms_out, int64_t* count_out);

/*
 * Test hook (the paper has no counterpart): make a later host allocation of object
 * construction fail. after >= 0 arms a countdown over the library's host allocation points
 * (plan, multi-rate plan and batch construction): the point that finds it at zero fails as an
 * out-of-memory allocation would, so that call returns SND_ERR_NOMEM and creates nothing; the
 * hook then disarms itself. after < 0 disarms it. Process-wide; returns SND_OK.
 */
int snd_debug_fail_host_alloc(int32_t after);

/*
 * Test hook (the paper has no counterpart): shrink the bounds of this plan's bounded device
 * loops. `limit` bounds the iteration loops (the union-find walks and the matched filter's
 * threshold search, in steps); `wait_cycles` bounds the waits (the tree's and the matched
 * filter's staging waits and the many-beam candidate stage's grid barrier, in clock cycles; a
 * batch uses its first plan's bound for the barrier). A loop that reaches its bound sets a
 * device status bit and the kernel returns (a staging wait that gives up still waits, with the
 * normal bound, for its copies in flight); snd_candidates then returns SND_ERR_TIMEOUT and
 * snd_plan_stats shows the bits. 0 restores the default of either bound; negative values are
 * SND_ERR_ARG. Rebinding the workspace clears the status word.
 */
int snd_debug_loop_limit(snd_plan_t plan, int64_t limit, int64_t wait_cycles);

/*
 * Encoder without device allocation (the paper has no counterpart: this is a convenience for
 * callers that cannot allocate device memory, e.g. code running where cudaMalloc is not
 * allowed or plugins that are handed only pre-allocated buffers). Encodes one chunk on its
 * own (statistics over this chunk, samples counted from its first row) exactly as
 * snd_execute's encoder does:
 *   d_chunk     device uint8[nsamp][nchan], read only
 *   theta       encoder threshold in sigma (snd_options_t.enc_theta)
 *   d_bits_out  device uint32[nchan][ceil(nsamp/32)]: bit i of word w is x_c(32 w + i)
 * Needs no workspace: its histogram scratch is a static device array sized for at most 4096
 * channels; nchan > 4096 or nsamp > 16,776,960 (= 65535 x 256) returns SND_ERR_UNSUPPORTED
 * before any work is enqueued. The first call on a device looks the array up and must come
 * before any stream capture. Calls on one device share the array, so calls that overlap on
 * the GPU race; serialise them. No allocation is made. Launch errors are checked after every
 * launch (SND_ERR_CUDA); a launch error left pending by earlier work on the calling thread is
 * reported, and cleared, the same way.
 */
int snd_encode_static(const uint8_t* d_chunk, int32_t nsamp, int32_t nchan, double theta, uint32_t* d_bits_out,
                      void* stream);

/* Release the plan's host memory. The workspace is the caller's. NULL is ignored. */
void snd_destroy(snd_plan_t plan);

/*
 * Multi-rate search (Methods, "Multi-rate extension"; Eq. scrunch). Each trial DM d runs at
 * the scrunch factor S(d) = the largest power of two, at most s_max, with
 * S*dt <= K d df / f_c^3 (df = |f_1 - f_0|, f_c = (max f + min f)/2, MHz). The DMs that share
 * one S form a band, searched by its own plan (same mode, options and branching) at sample
 * interval S*dt on the chunk averaged over S samples, (sum + S/2)/S per channel in uint8.
 * Band candidates are reported in native units (t * S, width * S) with the global DM index
 * and merged by single linkage: candidates within 20 pc cm^-3 and 200 ms of one another
 * (through any chain) form one cluster, reported by its largest S/N (ties: smaller DM index,
 * then smaller t), the list sorted by (t, dm_index).
 *   opts       options of every band (NULL: Table S1 of `mode`); each band plan gets
 *              max_chunk / S as its own max_chunk. opts->max_chunk must be a multiple of the
 *              largest S in use (else SND_ERR_ARG)
 *   s_max      largest scrunch factor, a power of two in 1..1024
 * Errors: SND_ERR_ARG, SND_ERR_DM, SND_ERR_NOMEM and whatever snd_plan_ex returns for a band.
 */
typedef struct snd_multirate_s* snd_multirate_t;
int snd_multirate_plan(const double* freqs_mhz, int32_t nchan, double dt_s, const double* dm_grid, int32_t ndm,
                       int32_t branching, snd_mode_t mode, const snd_options_t* opts, int32_t s_max,
                       snd_multirate_t* out);
/* Number of bands and, for the first `cap`, their scrunch factors and DM counts (either array
   may be NULL). Bands come in increasing S; a band's DMs keep the grid order. */
int snd_multirate_info(snd_multirate_t mr, int32_t* nbands, int32_t* scrunch, int32_t* band_ndm, int32_t cap);
/* The plan of band `band` (owned by `mr`: do not bind, execute or destroy it; statistics and
   profiling calls are allowed). */
int snd_multirate_band_plan(snd_multirate_t mr, int32_t band, snd_plan_t* out);
/* Device workspace bytes: every band plan's workspace, scrunch staging and the merge lists. */
size_t snd_multirate_workspace_size(snd_multirate_t mr);
/* Bind a 256-byte aligned workspace and reset every band's stream state; synchronises `stream`. */
int snd_multirate_bind_workspace(snd_multirate_t mr, void* d_workspace, size_t bytes, void* stream);
/* Next chunk, device uint8[nsamp][nchan]; nsamp a multiple of the largest S in use, at most
   max_chunk (else SND_ERR_CHUNK). Enqueued on `stream`, no host synchronisation. */
int snd_multirate_execute(snd_multirate_t mr, const uint8_t* d_chunk, int32_t nsamp, void* stream);
/* Replay each chunk's work (scrunching and every band's stages) as one CUDA graph, updated
   in place from chunk to chunk (enable != 0), or launch it directly (0, the default). */
int snd_multirate_set_graph(snd_multirate_t mr, int32_t enable);
/* Same for a host chunk, copied into the workspace first (cudaMemcpyAsync on `stream`). */
int snd_multirate_execute_host(snd_multirate_t mr, const uint8_t* h_chunk, int32_t nsamp, void* stream);
/* Merge the candidates of all bands found since the previous call (on the GPU), copy at most
   cap of them to host_out and clear the band lists; synchronises. SND_ERR_OVERFLOW and
   SND_ERR_TIMEOUT as for snd_candidates. */
int snd_multirate_candidates(snd_multirate_t mr, snd_candidate_t* host_out, int32_t cap, int32_t* n_out);
/* Release the band plans and host memory; NULL is ignored. */
void snd_multirate_destroy(snd_multirate_t mr);

/* Static description of a status code. */
const char* snd_error_string(int status);

/*
 * Many beams per step. A batch groups bound plans (one per beam; any mix of DM grids, chunk
 * lengths and options; the batch does not own them) and advances every beam by one chunk
 * per call, exactly as one snd_execute per beam would (same planes, same candidates; read
 * them with snd_candidates on each plan). Trees of beams whose plans share a kernel
 * instantiation run in one launch. With graphs enabled the step is captured on `stream` and
 * replayed as one CUDA graph, updated in place from step to step.
 *   d_chunks[i]  device uint8[nsamp[i]][nchan_i] chunk of beam i (host array of pointers)
 *   nsamp[i]     1..max_chunk of plan i
 * Plans with per-stage profiling enabled are rejected (SND_ERR_STATE); errors as snd_execute.
 */
typedef struct snd_batch_s* snd_batch_t;
int snd_batch_create(const snd_plan_t* plans, int32_t nplans, snd_batch_t* out);
int snd_batch_set_graph(snd_batch_t batch, int32_t enable);
int snd_batch_execute(snd_batch_t batch, const uint8_t* const* d_chunks, const int32_t* nsamp, void* stream);
/* Graph instantiations and in-place updates so far. */
int snd_batch_graph_stats(snd_batch_t batch, int64_t* instantiations, int64_t* updates);
void snd_batch_destroy(snd_batch_t batch);

/*
 * Learned candidate sifter (the paper leaves a learned classifier to future work,
 * "Discussion"; the plain threshold-and-clustering sifter above stays the default and the
 * reference). A CNN classifies 64-DM x 256-sample snippets of the float plane around
 * candidates: three 3x3 convolutions (16/32/64 channels, zero padding 1, bias, ReLU), each
 * followed by 2x2 max pooling, then fc 16384 -> 128 (ReLU) and fc 128 -> 1 (the logit of
 * "astrophysical"). Loss: mean binary cross-entropy. Parameters: one FP32 vector of
 * snd_sifter_num_params() values, in the order W1[16][1][3][3], b1[16], W2[32][16][3][3],
 * b2[32], W3[64][32][3][3], b3[64], Wf1[128][16384] (features c*256 + y*32 + x), bf1[128],
 * Wf2[128], bf2[1]. Convolutions and fc1 run as BF16 tensor-core GEMMs with FP32
 * accumulation (forward and backward); training uses Adam (beta 0.9 / 0.999, eps 1e-8).
 * Snippets are FP32 [n][64][256]; labels FP32 0/1 [n]. All device pointers; calls enqueue
 * on `stream` (snd_sifter_gradients and snd_sifter_status synchronise it).
 */
typedef struct snd_sifter_s* snd_sifter_t;
/* Host only. max_batch: largest n of any call (1..65536); training != 0 also sizes the
   backward and optimizer buffers; seed: He-uniform initial weights (zero biases). */
int snd_sifter_create(int32_t max_batch, int32_t training, uint64_t seed, snd_sifter_t* out);
int64_t snd_sifter_num_params(void);
size_t snd_sifter_workspace_size(snd_sifter_t sf);
/* Bind a 256-byte aligned device workspace and upload the initial parameters (synchronises). */
int snd_sifter_bind_workspace(snd_sifter_t sf, void* d_workspace, size_t bytes, void* stream);
/* Replace the parameters from host memory (n = snd_sifter_num_params()); resets Adam. */
int snd_sifter_set_params(snd_sifter_t sf, const float* host_params, int64_t n, void* stream);
int snd_sifter_get_params(snd_sifter_t sf, float* host_params, int64_t n);
/* Logits d_logits[n] of snippets d_x[n][64][256]. */
int snd_sifter_forward(snd_sifter_t sf, const float* d_x, int32_t n, float* d_logits, void* stream);
/* Loss (d_loss[1]) and its gradient with respect to every parameter (d_grads, num_params
   floats) on n labelled snippets, without an update (training plans only). Either output
   may be NULL. Synchronises; SND_ERR_TIMEOUT if a bounded device wait gave up. */
int snd_sifter_gradients(snd_sifter_t sf, const float* d_x, const float* d_y, int32_t n, float* d_grads,
                         float* d_loss, void* stream);
/* One Adam step of learning rate lr on n labelled snippets; d_loss (optional) receives the
   step's loss before the update. */
int snd_sifter_train_step(snd_sifter_t sf, const float* d_x, const float* d_y, int32_t n, float lr, float* d_loss,
                          void* stream);
/* Synchronise and report the device error word (SND_ERR_TIMEOUT) or a sticky error. */
int snd_sifter_status(snd_sifter_t sf);
/* CUDA kernels enqueued by this sifter so far. */
int64_t snd_sifter_launches(snd_sifter_t sf);
void snd_sifter_destroy(snd_sifter_t sf);

/*
 * Snippet extraction: d_out[i][64][256] = the float plane d_plane[ndm][ld] (ncols valid
 * columns) at rows d_rows[i] - 32 .. + 31 and columns d_cols[i] - 128 .. + 127, standardised
 * with the FP64 mean and population std of the cells inside the plane (std 0 -> 1); cells
 * outside are 0.
 */
int snd_snippets(const float* d_plane, int64_t ld, int32_t ndm, int64_t ncols, const int32_t* d_rows,
                 const int64_t* d_cols, int32_t n, float* d_out, void* stream);

/*
 * The sifter's tensor-core GEMM, exposed for testing: d_c[m][ldc] (FP32) = A . B^T with
 * A = d_a[m][lda] and B = d_b[n][ldb] BF16 row-major, k columns used (lda, ldb multiples of
 * 8, pointers 16-byte aligned). splits > 1 splits K over CTAs and ADDS into d_c (zero it
 * first). d_err: a device uint32 that receives a nonzero value if a bounded wait gave up.
 */
int snd_gemm_bf16(const void* d_a, int64_t lda, const void* d_b, int64_t ldb, int32_t m, int32_t n, int64_t k,
                  float* d_c, int64_t ldc, int32_t splits, uint32_t* d_err, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SND_H */
