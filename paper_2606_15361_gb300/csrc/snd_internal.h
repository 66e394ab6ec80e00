// Internal declarations shared by the host runtime and the CUDA kernels of the SND library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/snd.h"

namespace snd {

constexpr int kMaxLevels = 24;     // tree levels (leaves included) supported by the plan
constexpr int kNumWidthSlots = 11; // widths 1,2,4,...,1024 -> bit j of a row's width mask = 2^j
constexpr int kTreeThreadsPerDm = 32;
constexpr int kFlagReferenceTree = SND_FLAG_REFERENCE_TREE;

// Device status word bits (written by kernels, read by snd_candidates).
enum : uint32_t {
  kStatusCellOverflow = 1u << 0,
  kStatusRunOverflow = 1u << 1,
  kStatusCandOverflow = 1u << 2,
  kStatusBlockCandOverflow = 1u << 3,
  kStatusTauTimeout = 1u << 4,
  kStatusUnionTimeout = 1u << 5,
  kStatusBounds = 1u << 6,
  kStatusTreeTimeout = 1u << 7,
  kStatusGridTimeout = 1u << 8,
  kStatusMfTimeout = 1u << 9,
};

// One matched-filter cell kept for peak selection.
struct MfCell {
  uint32_t cell;   // row * nb + t (t relative to the block start)
  float snr;       // S/N rounded to float
  int32_t width;   // boxcar width of the cell's maximum
};

// Tree kernel shape: warps per CTA, trial DMs per warp, 32-sample words per lane.
struct TreeShape {
  int warps, dpw, kw;
};

// Tree kernel geometry (chosen on the host).
struct TreeGeom {
  int warps;           // warps per CTA
  int dpw;             // trial DMs per warp
  int kw;              // 32-sample words per lane
  int dms_per_cta;     // warps * dpw
  int tile_words;      // largest output words per CTA (32 * kw)
  int group_leaves;    // leaves staged per shared-memory round (a multiple of B)
  int span;            // words of one staged leaf-pattern series (per plane)
  int cspan;           // words of one staged channel window
  int max_pat_group;   // max pattern entries in one group of one DM tile
  int planes;          // planes of a leaf value (1 binary, 3 graded/float)
  int smem_bytes;      // dynamic shared memory per CTA
  int ndm_tiles;
};

// Direct tree kernel (tree_direct.cu) instantiations.
enum {
  kDirNone = -1,
  kDirFloat11 = 0,   // float, counts < 2048, 4 words per lane
  kDirFloat13,       // float, counts < 8192
  kDirGraded9U1,     // graded, exact-level nodes of <= 511 channels, one capped level above
  kDirGraded9U2,     // graded, as above with two capped levels above (2 words per lane)
  kDirGraded11U0,    // graded, the exact level is the root (<= 2047 channels)
  kDirGraded13U0,    // graded, the exact level is the root (<= 8191 channels)
  kDirBinary4,       // binary, C = 4, <= 4 levels above the leaves
  kDirBinary8,       // binary, <= 8 levels above the leaves
  kDirBinary12,      // binary, <= 12 levels above the leaves (2 words per lane)
  kDirBinReg4K1,     // binary, regular tree B = 4, K_I = 1, <= 4 levels above level 2
  kDirBinReg4K2,     // binary, regular tree B = 4, K_I = 2
  kDirBinReg8K1,     // binary, regular tree B = 8, K_I = 1, <= 3 levels above level 1
  kDirBinReg8K2,     // binary, regular tree B = 8, K_I = 2
  kDirBinReg2K1,     // binary, regular tree B = 2, K_I = 1, <= 4 levels above level 4
  kDirBinReg2K2,     // binary, regular tree B = 2, K_I = 2
};

// Direct tree kernel geometry: CTA = 32 consecutive trial DMs (lane = DM) x warps * kw words.
struct DirectGeom {
  int inst = kDirNone;
  int warps = 8;
  int kw = 4;
  int tile_words = 32;   // warps * kw
  int ndm_tiles = 0;     // ceil(ndm / 32)
  int cspan = 0;         // staged ring words per channel (multiple of 4)
  int sgroups = 1;       // 64-channel adder groups staged per round (1 or 2)
  int smem_bytes = 0;
  int sub_lev = 0;       // graded: the exact level (first level whose nodes may exceed N)
  int sub_groups = 1;    // graded: 64-channel groups per exact-level node
  int rates_inst = kDirNone;  // float / graded with per-level fire counts: the binary counting pass
  int rates_kw = 4;
};

// Labelled-payload (zfloat) tree geometry (chosen on the host).
struct ZGeom {
  int fp16;           // payload and partial sums stored in FP16 (else FP32)
  int unit;           // payload 1 for every spike (the paper's 0/1 raster) instead of z
  int maxl;           // level capacity of the kernel instantiation (4, 8, 16)
  int spt;            // output samples per lane
  int dms_per_cta;    // DM rows per CTA (one warp each)
  int tile_samples;   // output samples per CTA (32 * spt)
  int ndm_tiles;
  int win;            // staged payload samples per channel
  int group_leaves;   // leaves staged per shared-memory round
  int smem_bytes;
  int Rz;             // payload ring samples per channel
};

// Device pointers inside the bound workspace.
struct DevPtrs {
  uint32_t* ring;          // [nchan][2R] bit ring (mirrored)
  uint32_t* hist;          // [nchan][256]
  int32_t* levels;         // [nchan] encoder level u_c (256 = never)
  int32_t* plane;          // [ndm][Lp] root values by absolute time modulo Lp
  uint32_t* mask;          // [ndm][mw] matched-filter mask of the current block
  uint32_t* mask2;         // [ndm][mw] closing scratch
  uint32_t* mask3;         // [ndm][mw] closed mask
  MfCell* cells;           // [cell_cap]
  uint32_t* counters;      // [16] misc counters (cells, runs, block cands, cands, status ...)
  int32_t* row_runs;       // [ndm + 1] run offsets per row (exclusive scan)
  int32_t* run_start;      // [run_cap]
  int32_t* run_end;        // [run_cap]
  int32_t* run_row;        // [run_cap]
  int32_t* parent;         // [run_cap]
  int32_t* npix;           // [run_cap]
  unsigned long long* peak;// [run_cap]
  int32_t* pwidth;         // [run_cap] width of the island's peak cell
  snd_candidate_t* bcand;  // [cand_cap] candidates of the current block (unsorted)
  snd_candidate_t* cand;   // [cand_cap] accumulated sorted candidates
  uint8_t* staging;        // [max_chunk * nchan] host-chunk staging (two buffers, used in turn)
  uint8_t* staging2;       // [max_chunk * nchan]
  // plan tables
  uint16_t* width_mask;    // [ndm]
  float* dm_f32;           // [ndm]
  int32_t* tp_off;         // [ndm_tiles * nleaves + 1]
  uint32_t* gepk;          // [ntp * C] staged-window word offset << 5 | shift per entry channel
  int32_t* gleaf;          // [ntp] leaf of each entry relative to its group
  uint32_t* gmeta;         // [ndm * nleaves] series word offset << 5 | shift per (DM, leaf)
  int32_t* tile_wb;        // [ndm_tiles * nchan] first staged ring word per channel (tile-relative)
  int32_t* delays;         // [ndm * nchan] full delay table (reference kernel, tests)
  void* zring;             // zfloat: [nchan][Rz] payload ring (half or float), sample a at a mod Rz
  void* ztab;              // zfloat: [nchan][256] payload of each uint8 value (0 below the level)
  int32_t* zwb;            // zfloat: [ndm_tiles][nchan] first staged sample offset per channel
  int32_t* zcarry;         // zfloat: [nleaves] carry depth of each leaf
  uint16_t* dmeta;         // direct tree: [ndm_tiles][nchan][32] staged word offset << 5 | shift
  int32_t* dbase;          // direct tree: [ndm_tiles][nchan] first staged ring word (multiple of 4)
  unsigned long long* level_fires;  // [kMaxLevels] firing node-samples per tree level (SND_FLAG_LEVEL_RATES)
};

// Counter slots.
enum {
  kCntCells = 0,
  kCntRuns = 1,
  kCntBlockCands = 2,
  kCntCands = 3,
  kCntStatus = 4,
  kCntTreeQueue = 8,   // many-beam tree: next work item (the first plan of a batch launch)
  kCntGridBar = 12,    // many-beam candidates: grid barrier arrivals, generation (two slots)
  kCntSlots = 16
};

struct Plan {
  // configuration
  int nchan = 0, ndm = 0, mode = 0, B = 2, C = 4, KL = 2, KI = 2, N = 255;
  double dt = 0, enc_theta = 1.5, det_theta = 7.0, sigma_min = 0.2, mf_alpha = 0.1;
  int closing = 9, n_min = 10, max_chunk = 32768, cand_cap = 65536, cell_cap = 1 << 20,
      run_cap = 1 << 21, flags = 0, plane_u8 = 0, tree_warps = 0, tree_round = 0;
  std::vector<double> freqs, dms;

  // derived
  int ref_chan = 0, min_chan = 0;
  int D = 0;
  std::vector<int32_t> delays;          // [ndm][nchan]
  std::vector<uint16_t> width_mask;     // [ndm]
  int wmax = 1;
  int nlev = 1;
  std::vector<int> level_nodes;         // nodes per level (leaves first)
  std::vector<int64_t> level_unique;    // distinct patterns per level
  double adds_per_dm_sample = 0;
  int64_t hist_mem_bytes = 0;
  int nleaves = 0;

  // leaf patterns and tiles
  int npat = 0;
  std::vector<int32_t> pat_rel;         // [npat][C]
  std::vector<int32_t> leaf_pid;        // [ndm][nleaves]
  std::vector<int32_t> tp_off, tp_pid, tp_smin, tp_leaf;
  std::vector<uint8_t> dl_lp;
  std::vector<int32_t> dl_sh;
  std::vector<int32_t> tile_wb;
  std::vector<uint32_t> gepk, gmeta;  // precomputed staging offsets (see choose_tree_geometry)
  std::vector<int32_t> gleaf;
  TreeGeom geom{};
  DirectGeom dgeom{};
  bool direct = false;                  // the tree runs on the direct kernel (tree_direct.cu)
  std::vector<uint16_t> dmeta;
  std::vector<int32_t> dbase;
  ZGeom zgeom{};
  std::vector<int32_t> zwb, zcarry;

  // sizes
  int R = 0;           // ring words per copy
  int Lp = 0;          // plane ring columns (multiple of 32)
  int mw = 0;          // mask words per row
  size_t ws_bytes = 0;
  struct Off {
    size_t ring, hist, levels, plane, mask, mask2, mask3, cells, counters, row_runs, run_start,
        run_end, run_row, parent, npix, peak, pwidth, bcand, cand, staging, staging2, width_mask, dm_f32, tp_off,
        gepk, gleaf, gmeta, tile_wb, delays, zring, ztab, zwb, zcarry, dmeta, dbase, level_fires;
  } off{};

  // binding and stream state
  void* ws = nullptr;
  size_t ws_have = 0;
  DevPtrs dp{};
  bool bound = false;
  cudaStream_t last_stream = nullptr;
  int64_t T = 0;   // samples consumed
  int64_t E = 0;   // emitted plane samples
  int64_t F = 0;   // scored start times
  int sticky = 0;
  int pending_host = -1;
  int64_t loop_limit = 0;        // test hook: bound of the iteration loops (0 = defaults)
  int64_t wait_limit = 0;        // test hook: bound of the waits, clock cycles (0 = defaults)
  uint32_t last_status = 0;      // device status word read by the last snd_candidates
  mutable int64_t launches = 0;  // kernels enqueued since binding

  // host-chunk uploads (snd_execute_host): the two staging buffers are filled in turn on a
  // private copy stream, so chunk i+1's copy overlaps chunk i's kernels
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_done[2] = {nullptr, nullptr};  // copy into buffer b finished
  cudaEvent_t up_free[2] = {nullptr, nullptr};  // the chunk that read buffer b finished
  bool up_free_set[2] = {false, false};
  int up_next = 0;

  // per-stage timing (snd_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;       // created on demand, reused
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;  // (stage, (start, stop))
  ~Plan();
};

// plan.cpp
int build_plan(Plan& p);
// A host allocation point of object construction: throws std::bad_alloc when the failure
// injection of snd_debug_fail_host_alloc reaches it (callers map that to SND_ERR_NOMEM).
void alloc_point();

// runtime.cu: the positions of one chunk (Methods, "Pipeline overview", ring-buffer form):
// plane samples [e_prev, e_new) are emitted, start times [f_prev, f_new) scored (nb of them)
struct ChunkPos {
  int64_t e_prev, e_new, f_prev, f_new;
  int nb;
};
ChunkPos chunk_pos(const Plan& p, int32_t nsamp);
void chunk_commit(Plan& p, const ChunkPos& c, int32_t nsamp, cudaStream_t s);

// Matched filter and candidate stages of a chunk whose tree has run; `stage(id, f)` runs the
// launcher f (optionally timed).
template <typename Stage>
cudaError_t chunk_post(const Plan& p, const ChunkPos& c, void* d_plane_out, cudaStream_t s, Stage&& stage);

// kernels (launchers), each returns cudaGetLastError() of its launch and adds the number
// of kernels it enqueued to p.launches
cudaError_t launch_encode(const Plan& p, const uint8_t* d_chunk, int nsamp, cudaStream_t s);
cudaError_t launch_tree(const Plan& p, int64_t e_prev, int64_t e_new, cudaStream_t s);
cudaError_t launch_mf(const Plan& p, int64_t e_prev, int64_t e_new, int64_t f_prev, int64_t f_new,
                      void* d_plane_out, cudaStream_t s);
cudaError_t launch_candidates(const Plan& p, int64_t f_prev, int nb, cudaStream_t s);
// many-beam launchers (encode.cu, mf.cu, ccl.cu): several plans' chunk stages in few launches
cudaError_t launch_encode_batch(const Plan* const* plans, const uint8_t* const* chunks, const int32_t* nsamp, int n,
                                cudaStream_t s);
cudaError_t launch_mf_batch(const Plan* const* plans, const ChunkPos* pos, int n, cudaStream_t s);
cudaError_t launch_candidates_batch(const Plan* const* plans, const ChunkPos* pos, int n, cudaStream_t s);
TreeShape tree_shape(int mode, int nlev, int kmax);  // k_tree launch shape
cudaError_t launch_tree_batch(const Plan* const* plans, const int64_t* e_prev, const int64_t* e_new, int n,
                              cudaStream_t s);
// batch.cu: one chunk of each plan (all encoders, the trees, all matched filters and all
// candidate stages, each in a few launches), enqueued on s; the plans then record `owner` as
// their stream
int enqueue_plans(Plan* const* plans, int n, const uint8_t* const* d_chunks, const int32_t* nsamp, cudaStream_t s,
                  cudaStream_t owner);

// Replays enqueued work as a CUDA graph: captured on a private stream, updated in place from
// call to call while the topology is unchanged, launched on the caller's stream.
struct GraphRunner {
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t instantiations = 0, updates = 0;
  int run(cudaStream_t s, const std::function<int(cudaStream_t)>& enqueue);
  ~GraphRunner();
};

cudaError_t launch_tree_z(const Plan& p, int64_t e_prev, int64_t e_new, void* d_plane_out, cudaStream_t s);
// tree_direct.cu: the direct tree kernel of plans with p.direct
cudaError_t launch_tree_direct(const Plan& p, int64_t e_prev, int64_t e_new, cudaStream_t s);
cudaError_t launch_tree_direct_batch(const Plan* const* plans, const int64_t* e_prev, const int64_t* e_new, int n,
                                     cudaStream_t s);

template <typename Stage>
cudaError_t chunk_post(const Plan& p, const ChunkPos& c, void* d_plane_out, cudaStream_t s, Stage&& stage) {
  cudaError_t e = cudaSuccess;
  if (c.nb > 0) e = cudaMemsetAsync(p.dp.counters, 0, sizeof(uint32_t) * (kCntBlockCands + 1), s);
  if (e == cudaSuccess && (c.nb > 0 || (d_plane_out && c.e_new > c.e_prev)))
    e = stage(SND_STAGE_MF, [&] { return launch_mf(p, c.e_prev, c.e_new, c.f_prev, c.f_new, d_plane_out, s); });
  if (e == cudaSuccess && c.nb > 0)
    e = stage(SND_STAGE_CANDIDATES, [&] { return launch_candidates(p, c.f_prev, c.nb, s); });
  return e;
}

}  // namespace snd
