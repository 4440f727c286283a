// internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <map>
#include <mutex>
#include <utility>

#include <cstdint>
#include <cuda_runtime.h>

// The context behind the opaque sws_ctx handle of the C ABI.
struct sws_ctx {
  int device = 0;
  int *d_err = nullptr;  // device error word (DevErr bits)
  void *ws = nullptr;    // workspace
  uint64_t ws_size = 0;
  int num_sms = 0;
  // sliding-sum variants chosen by sws_tune_sliding_sum, per (operator, w): variant and the n
  // it was timed on
  std::mutex tune_mu;
  struct Tuned {
    int variant, shape;
    uint64_t n;
  };
  std::map<std::pair<int, int>, Tuned> tuned;
};

namespace sws {

// Tile configurations of the sliding-sum kernels: threads per CTA x elements per thread.
enum SlideCfg { CFG_SMALL = 0, CFG_LARGE = 1, CFG_COUNT = 2 };

struct SlideLaunch {
  int op;       // SWS_OP_*
  int variant;  // SWS_VARIANT_*
  int cfg;      // SlideCfg
  int num_sms;  // SMs of the device (grid of the persistent kernel)
  int *err;     // device error word (bounded waits)
  int shape = 0;  // warp-private runs: 0 = chosen by block width, 1..3 = a fixed run shape
};
constexpr int kWarpShapes = 3;

// Tile length (elements) of a configuration for elements of `esize` bytes.
int slide_tile_len(int cfg, int esize);
// Outputs per tile, or 0 when w does not fit the configuration.
int slide_tile_outputs(int cfg, int esize, int w);

// Fill `bytes` of device memory with a fixed pseudo-random pattern (timing inputs).
cudaError_t launch_fill_pattern(void *dst, uint64_t bytes, cudaStream_t stream);

// Queue one sliding sum; the caller has validated the arguments.
cudaError_t launch_sliding_sum(const SlideLaunch &L, const void *in, void *out, uint64_t n, int w,
                               cudaStream_t stream);

// Minimizer kernel parameters (one launch covers one sequence or one read batch).
struct MiniArgs {
  const uint8_t *seq;    // packed DNA (source DNA)
  const uint32_t *keys;  // precomputed keys (source KEYS)
  uint64_t n;            // bases or keys
  int k, w, mode;
  const int64_t *bar;    // N-block pairs, or read offsets (nreads + 1) in batch mode
  uint64_t nbar;         // number of N-blocks, or number of reads
  void *hash_out;
  uint32_t *pos_out;
  uint64_t capacity;
  uint64_t *count_out;
  uint64_t *pick_offsets;  // batch mode: [nreads + 1]
  // workspace
  unsigned long long *status;  // one word per tile, zeroed before the launch
  unsigned int *tile_counter;  // zeroed before the launch
  uint2 *tile_bar;             // one word per tile (filled by the launcher when barriers exist)
  int *err;                    // device error word of the context
  // staged path only
  uint32_t *tile_counts;  // [num_tiles + 1], exclusive offsets after the scan
  uint32_t *scan_tmp;     // scan_u32_scratch_words(num_tiles + 1)
  void *stg_hash;         // [num_tiles * windows per tile] values, mini_fast_hash_bytes each
  uint32_t *stg_pos;
  uint32_t *stg_first;    // read batches: read index of a read's first pick, else ~0
  // When set, the sizes (n, nbar, windows, tiles) are read from this device descriptor at run
  // time instead of from the fields above: one captured graph then serves any batch up to the
  // sizes it was built for.  Layout: see BatchDesc.
  const unsigned long long *desc;
  // Failure self-test only: the look-back kernel announces its staging copies but never issues
  // them, so every tile's bounded copy wait runs out.
  int withhold_copy;
  // Staged path: count the picks only (no staging area; the total goes to count_out).
  int count_only;
};

// Device descriptor of a batch, read by the kernels of a captured batch graph.
enum BatchDesc { BD_NREADS = 0, BD_TOTAL = 1, BD_NWIN = 2, BD_TILES = 3, BD_SCAN_LEN = 4, BD_WORDS = 8 };

enum MiniSource { SRC_DNA = 0, SRC_KEYS = 1 };
enum MiniBarrier { BAR_NBLOCK = 0, BAR_READS = 1 };

// Look-back path (any w <= 4000, any k): one kernel, picks placed in order by a decoupled
// look-back over per-tile status words (zeroed, with the tile counter, before the launch).
int mini_tile_windows(int w);  // windows per tile (a multiple of 64), 0 if w is too large
uint64_t mini_lookback_tiles(uint64_t nwin, int w);
cudaError_t launch_minimizers_lookback(const MiniArgs &a, int source, int barrier, uint64_t num_tiles,
                                       cudaStream_t stream);
// Staged path (w in 4..256, k-mers of at most 32 bases or precomputed keys): a persistent kernel
// writes each tile's picks to a fixed slot, a scan of the per-tile counts gives offsets, a gather
// puts picks in order.
bool mini_fast_applies(int source, int k, int w);
int mini_fast_hash_bytes(int source, int k);  // bytes of a staged key value: 8 when 2k > 32
// Windows per tile of the staged path: the specialised kernel's for w in 4..256, else the generic
// kernel's (which then runs in staged mode).
int mini_staged_tile_windows(int source, int k, int w);
cudaError_t launch_minimizers_generic_staged(const MiniArgs &a, int source, int barrier, uint64_t num_tiles,
                                             const uint2 *tile_bar, cudaStream_t stream);
int mini_fast_tile_windows(int w);
cudaError_t launch_minimizers_staged(const MiniArgs &a, int source, int barrier, uint64_t num_tiles,
                                     cudaStream_t stream);

// Sliding minimum over precomputed keys for w <= 17 (keys_min.cu): one pass, picks placed in
// order by per-tile counts.  Needs keys aligned to 16 bytes and at least 32 of them.
bool keys_min_applies(const uint32_t *keys, uint64_t m, int w);
uint64_t keys_min_ws_bytes(uint64_t m, int w);  // workspace (zeroed by the launcher)
cudaError_t launch_keys_min(const uint32_t *keys, uint64_t m, int w, uint32_t *key_out, uint32_t *pos_out,
                            uint64_t capacity, uint64_t *count_out, void *ws, int *err, int num_sms,
                            cudaStream_t stream);
// The same kernel on hashed canonical k-mers of a packed sequence (k <= 29, 4 <= w <= 17, the
// sequence 4-byte aligned; 64-bit keys above k = 16): each thread hashes its 16 k-mers in
// registers.  Barriers: none,
// N-blocks (barrier BAR_NBLOCK, nbar pairs), or the read starts of a batch (BAR_READS, nbar reads,
// positions read-local, each read's first pick index in pick_offsets, which the caller sets to
// all ones first and fixes up after).  With desc the sizes come from a batch descriptor and
// n is the batch's capacity.  Workspace: dna_min_ws_bytes(n, k, w).
struct DnaMinArgs {
  const uint8_t *seq;
  uint64_t n;
  int k, w;
  int barrier;  // -1: none
  const int64_t *bar;
  uint64_t nbar;
  uint64_t *pick_offsets;
  const unsigned long long *desc;
  uint32_t *key_out, *pos_out;
  unsigned long long *key_out64;  // the keys when k > 16
  uint64_t capacity;
  uint64_t *count_out;
};
bool dna_min_fits(uint64_t n, int k, int w, int mode);  // the sizes and mode allow it
bool dna_min_applies(const uint8_t *seq, uint64_t n, int k, int w, int mode);  // and seq is aligned
int dna_min_tile_windows();
uint64_t dna_min_ws_bytes(uint64_t n, int k, int w);
cudaError_t launch_dna_min(const DnaMinArgs &d, void *ws, int *err, int num_sms, cudaStream_t stream);

// The per-tile summary of the barriers (N-blocks or read starts) that can touch each tile.
bool tile_barriers_needed(const MiniArgs &a, int source, int barrier);
cudaError_t launch_tile_barriers(const MiniArgs &a, int source, int barrier, uint64_t num_tiles, int TW, int span,
                                 cudaStream_t stream);
// Exclusive scan of uint32 counts in place (scratch of scan_u32_scratch_words(len) words).
uint64_t scan_u32_scratch_words(uint64_t len);
cudaError_t scan_u32(uint32_t *a, uint64_t len, uint32_t *bsum, cudaStream_t stream);
// The same with the length read at run time from *dlen (at most max_len).
cudaError_t scan_u32_dev(uint32_t *a, uint64_t max_len, const unsigned long long *dlen, uint32_t *bsum,
                         cudaStream_t stream);
// Batch fix-up: reads without picks get the offset of the next read that has some.  With `desc`
// set, the number of reads is read from it at run time (nreads is then the maximum).
cudaError_t launch_pick_offsets_fixup(uint64_t *pick_offsets, uint64_t nreads, const uint64_t *count,
                                      uint64_t *scratch, cudaStream_t stream,
                                      const unsigned long long *desc = nullptr);
// k-mer values.
cudaError_t launch_kmers(const uint8_t *seq, uint64_t n, int k, int kind, void *out, int *err, cudaStream_t stream);

// Seed table (radix sort + pointer table).
struct TableArgs {
  const void *hash;       // uint32 (hash_bits <= 32) or uint64
  const uint32_t *pos;
  uint64_t m;
  int hash_bits, bucket_bits;
  void *sorted_hash;
  uint32_t *sorted_pos;
  uint64_t *offsets;      // 2^bucket_bits + 1
  // workspace
  unsigned long long *ws_keys[2];
  uint32_t *ws_vals[2];   // hash_bits > 32 only
  uint32_t *ws_hist;      // table_hist_words(m)
  uint32_t *ws_bsum;      // table_bsum_words(m)
  void *ws_gaps;          // table_gap_bytes(bucket_bits)
  unsigned long long *ws_ngaps;
  uint64_t gap_cap;
  void *ws_msd;  // table_msd_bytes(m): the segmented sort's descriptors (nullptr: LSD passes only)
};
uint64_t table_gap_capacity(int bucket_bits);
uint64_t table_hist_words(uint64_t m);
uint64_t table_bsum_words(uint64_t m);
uint64_t table_gap_bytes(int bucket_bits);
uint64_t table_msd_bytes(uint64_t m);
cudaError_t launch_table(const TableArgs &a, cudaStream_t stream);

// Seeding (seed.cu).
uint64_t seed_hit_tiles(uint64_t nq);  // 8 bytes of workspace each
cudaError_t launch_seed_lookup(const void *sorted_hash, int hash_bits, int bucket_bits, const uint64_t *offsets,
                               const void *query, uint64_t nq, uint64_t *first, uint32_t *count, cudaStream_t stream);
cudaError_t launch_seed_hits(const uint64_t *first, const uint32_t *count, uint64_t nq, uint32_t max_occ,
                             const uint32_t *sorted_pos, uint32_t *hit_query, uint32_t *hit_pos, uint64_t capacity,
                             uint64_t *hit_count, unsigned long long *tile_ws, cudaStream_t stream);

// Strands of minimizer picks (strand.cu).
cudaError_t launch_strands(const uint8_t *seq, uint64_t n, int k, const int64_t *base_offsets,
                           const uint64_t *pick_offsets, uint64_t nreads, const uint32_t *pos, uint64_t m,
                           uint8_t *strand, cudaStream_t stream);

// Error reporting and argument checks shared with api.cu (sws_status is an int).
int report_error(int status, const char *msg);
int check_minimizer_args(int k, int w, int mode);

// Device error bits.
enum DevErr { DEVERR_LOOKBACK_TIMEOUT = 1, DEVERR_COPY_TIMEOUT = 2 };

// One warp running a bounded wait on a flag nothing sets (0: look-back poll on `status`, two
// zeroed words; 1: an mbarrier expecting bytes that never arrive); records the time-out in err.
cudaError_t launch_selftest_wait(int which, unsigned long long *status, int *err, cudaStream_t st);

}  // namespace sws
