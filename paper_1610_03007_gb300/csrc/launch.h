// Host-side launchers of the gbsa kernels (one .cu file per step of the
// method). All launches are asynchronous on `stream`.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbsa.h"
#include "common.cuh"

namespace gbsa {

// ---- runtime helpers (engine.cu) ----------------------------------------
// SM count of the current device, cached per device; thread-safe.
int device_sm_count();
// Allows `smem_bytes` of dynamic shared memory for kernel `fn` (and, with
// max_carveout, the largest shared-memory carveout), once per kernel and
// CUDA context: function attributes belong to a context, so a process that
// launches on several GPUs, or again after cudaDeviceReset, must set them
// in each. Thread-safe; concurrent first calls may both set them (harmless).
cudaError_t ensure_smem_attributes(const void *fn, int smem_bytes, bool max_carveout);
// sa_build_ex; stage_readbacks false keeps every readback on the copy
// engine through pageable memory (no pinned host allocation, for
// sa_build_noalloc).
sa_status build_single(const uint8_t *text, uint64_t n, uint32_t *sa_out, uint32_t *isa_out,
                       void *workspace, size_t ws_bytes, const sa_options *opt, sa_stats *stats,
                       gbsa_stream_t stream, bool stage_readbacks);
// The tuning table's parameters for a build of this class (tuning.cu); all
// fields 0 when no entry applies.
void tuned_params(bool batched, uint32_t bits, uint64_t n, sa_tuned *out);

// Copies by kernels (k_gather.cu): dst/src may be pinned host memory
// (device-mapped), so the copy does not queue on a copy engine.
cudaError_t launch_copy_words(uint32_t *dst, const uint32_t *src, uint64_t words,
                              cudaStream_t stream);
cudaError_t launch_copy_bytes(uint8_t *dst, const uint8_t *src, uint64_t n, cudaStream_t stream);

// ---- step A0: alphabet (k_alphabet.cu) ----------------------------------
// hist[256] += occurrences of each byte value in text[0, n). hist must be
// zeroed by the caller.
cudaError_t launch_byte_histogram(const uint8_t *text, uint64_t n, uint32_t *hist,
                                  int num_sms, cudaStream_t stream);

// ---- step A1: initial keys (k_pack.cu) ----------------------------------
struct PackArgs {
  const uint8_t *text;     // concatenated texts
  uint32_t N;              // total characters
  const uint32_t *seg_off; // S+1 ungapped offsets (device)
  uint32_t S;              // number of texts
  const uint8_t *code;     // dense order-preserving code of each byte (device)
  uint32_t b;              // bits per character
  uint32_t c0;             // characters per key
  uint32_t cb;             // c0 * b (segment id sits above these bits)
  uint64_t *keys;          // out: N keys, tail-first order per text
  uint32_t *vals;          // out: N gapped positions
  DigitSpec spec;          // digits of the following radix sort
  uint32_t *hist;          // out: += their histograms (P * 256, zeroed by the caller)
  // 1: one text whose digits hold whole characters (b divides 8, cb a
  // multiple of 8, P = cb / 8): only the top digit is counted per key and
  // the other histograms are derived from it (k_pack_hist_fixup).
  uint32_t top_only;
};
// keys == NULL (top_only only): the histograms alone (the first radix pass
// then builds the keys from the text, PassArgs.text).
cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream);

// ---- step A2: radix sort (k_sort.cu) ------------------------------------
// hist[P*256] += digit counts of keys[0, m) for the digits in spec.
// rs (device-driven rounds): m and spec come from rs->mL and rs->spec
// instead (m then sizes the grid only).
cudaError_t launch_digit_histogram(const uint64_t *keys, uint32_t m, const DigitSpec &spec,
                                   uint32_t *hist, int num_sms, cudaStream_t stream,
                                   const RoundState *rs = nullptr);
// Exclusive digit offsets, constant-digit skipping and buffer ping-pong.
// keep_first: pass 0 is kept even if its digit is constant (it is the pass
// that reads the text, PassArgs.text).
cudaError_t launch_sort_plan(const uint32_t *hist, uint32_t *digit_base, const DigitSpec &spec,
                             uint32_t m, uint64_t *ka, uint64_t *kb, uint32_t *va,
                             uint32_t *vb, SortPlan *plan, Ctrl *ctrl, cudaStream_t stream,
                             const RoundState *rs = nullptr, bool keep_first = false);
// One stable one-sweep pass over digit p of the plan.
struct PassArgs {
  const SortPlan *plan;
  int p;
  uint32_t shift, bits;
  const uint32_t *digit_base;  // 256 entries for this pass
  uint32_t m;
  uint64_t *status;  // >= tiles * 256 words
  uint32_t epoch;
  uint32_t *tile_ctr;
  Ctrl *ctrl;
  uint32_t spin_limit;
  uint32_t inject;
  uint32_t items;    // keys per thread: 8, 12 or 16 (tile = 256 * items)
  // Device-driven rounds: sizes, digit and epoch base from the round state
  // (m then bounds the grid only; epoch is an offset). NULL: the fields above.
  const RoundState *rs;
  uint32_t grid_cap;  // at most this many blocks, each looping over tiles (0: one per tile)
  // Pass 0 of round 0 over one text (text != NULL, p == 0, not persistent):
  // the keys are built from the text in the layout of k_pack.cu (index j <
  // tails: the tail position n-1-j, zero-padded; j >= tails: position j -
  // tails) instead of read from the plan's source buffers.
  const uint8_t *text;
  const uint8_t *code;  // dense code of each byte (256 entries, device)
  uint32_t b, c0, cb, tails;
};
constexpr int SORT_TILE_MIN = 256 * 8;  // smallest tile (sizes the status array)
constexpr uint32_t SORT_ITEMS_DEFAULT = 16;
cudaError_t launch_onesweep(const PassArgs &a, cudaStream_t stream);
// Copies the plan's final buffer back to (ka, va) when it is buffer B.
cudaError_t launch_copy_back(const SortPlan *plan, uint64_t *ka, uint32_t *va, uint32_t m,
                             int num_sms, cudaStream_t stream);

// ---- steps A3+A4: rename, unique test, discard (k_rename.cu) ------------
struct RenameArgs {
  const SortPlan *plan;      // sorted keys / gapped positions
  uint32_t m;
  uint32_t round0;           // 1: initial naming with the end-of-text rules
  uint32_t cb;               // round 0: segment id = key >> cb (cb < 64)
  uint32_t c0;               // round 0: characters per key
  const uint32_t *seg_off;   // S+1 ungapped offsets
  uint32_t S;
  uint32_t W;                // later rounds: group ordinal g = key >> W
  // a-tuple rounds: {ka, kb}; the later partners of sorted position j are
  // in the buffer that does not hold the keys. {NULL, NULL} otherwise.
  const uint64_t *sec_buf[2];
  const uint32_t *base_in;   // later rounds: head rank - start of group g
  const uint32_t *old_in;    // later rounds: name of group g (round 0: NULL)
  uint32_t g_in;             // later rounds: groups in base_in (bounds guard)
  uint64_t *upd;             // queued ISA entries (head << 32 | i') of new unique suffixes
  uint32_t *isa;             // gapped ISA (not written; bounds of gapped positions)
  uint64_t isa_len;          // entries of isa (bounds guard)
  uint32_t N;                // total characters = entries of sa (bounds guard)
  uint32_t *sa;              // SA, written with indices local to each text
  uint64_t *act_out;         // survivors: (g' << 32) | i'
  uint32_t *gstart_out;      // start of each surviving group in act_out
  uint32_t *ghead_out;       // head rank (SA interval start) of each surviving group
  uint32_t *gold_out;        // name of its parent group (NO_NAME in round 0)
  const uint32_t *off_in;    // device: [survivor offset, group offset] of the output
  uint32_t *cnt_out;         // device: [survivors, groups] written by the last tile
  uint64_t *status;          // >= 2 * tiles words
  uint32_t epoch;
  uint32_t *tile_ctr;
  Ctrl *ctrl;
  uint32_t spin_limit;
  // Device-driven rounds: m = rs->mL, g_in = rs->GL and epoch base
  // rs->epoch (m above then bounds the grid only). NULL: the fields above.
  const RoundState *rs;
  uint32_t grid_cap;         // at most this many blocks, each looping over tiles (0: one per tile)
};
#ifndef GBSA_RN_ITEMS
#define GBSA_RN_ITEMS 8
#endif
constexpr int RENAME_TILE = 256 * GBSA_RN_ITEMS;
cudaError_t launch_rename(const RenameArgs &a, cudaStream_t stream);

// ---- rounds >= 1: small-group refine and large-group path (k_refine.cu) --
// Groups of up to REFINE_SMALL_MAX members are refined inside one tile
// (gather, shared-memory sort, rename, compaction); larger ones go through
// the global radix sort and k_rename.
// Tile shapes of the refine (threads per block, items one tile can hold).
// Tile t owns the groups whose starts fall in [t, t+1) * cap/2 of the
// active list, so groups of up to cap/2 members are "small".
struct RefineShape {
  uint32_t block, cap;
};
constexpr int REFINE_SHAPES = 4;
constexpr RefineShape REFINE_SHAPE[REFINE_SHAPES] = {{128, 1024}, {256, 2048}, {256, 4096},
                                                     {256, 1024}};
constexpr uint32_t REFINE_MIN_NOMINAL = 512;  // smallest cap/2 (buffer sizing)

// Names of groups. A name may be any rank inside the group's SA interval:
// intervals are disjoint and ordered, so such names respect the order of
// the suffixes, and a singleton's only choice is its rank. NAMES_HEAD is the
// paper's rule (Algorithm 5/6: the interval start, r + (subgroup start -
// group start)); NAMES_RETAIN keeps a parent's name in the subgroup whose
// interval contains it and gives every other subgroup the middle of its
// interval, so a majority subgroup keeps its name and fewer ISA entries
// change per round.
enum NamingRule : uint32_t { NAMES_HEAD = 0, NAMES_RETAIN = 1 };
constexpr uint32_t NO_NAME = 0xFFFFFFFFu;

struct ClassifyArgs {
  uint32_t *gstart;         // G entries written by this round; entry G set here
  uint32_t *gname;          // names: final for refine groups, set here for rename groups
  const uint32_t *ghead;    // head rank of every group
  const uint32_t *gold;     // parent names of the rename groups
  uint32_t naming;          // NamingRule
  uint32_t *lg, *loff, *lbase, *lold;  // large groups: index, start in the large
                                       // list, head - start, name
  uint32_t *tfirst;         // first group of each refine tile (tiles + 1 entries)
  uint32_t nominal;         // refine tile window (cap / 2); also the largest small group
  uint32_t max_groups;      // upper bound of G (buffer capacity)
  uint32_t max_tiles;       // upper bound of tiles (buffer capacity - 1)
  Ctrl *ctrl;               // reads rc.m_s + rc.m_l, rc.g_s + rc.g_l; adds to rc.large
  const RoundState *rs;     // device-driven rounds: nothing once the loop ended (else NULL)
};
cudaError_t launch_classify(const ClassifyArgs &a, int num_sms, cudaStream_t stream);

// keys[j] = (k << W) | r2 for the j-th item of the large groups, k = large
// group ordinal; vals[j] = gapped position. With a = 3 or 4 (a-tuples of
// names per round) instead keys[j] = the later partners (r3, or
// (r3 << W) | r4), vals[j] = j, and both keys are also kept by item in the
// stashes for k_wide_rekey / k_wide_finish.
struct GatherLargeArgs {
  const uint64_t *act;
  const uint32_t *gstart;
  const uint32_t *lg, *loff;
  uint32_t mL, GL;
  uint32_t h, W;
  uint32_t mult;            // a: 2, 3 or 4
  const uint32_t *isa;
  uint64_t isa_len;
  uint64_t *keys;
  uint32_t *vals;
  uint64_t *key1_stash;     // a > 2: (k << W) | r2 by item
  uint64_t *sec_stash;      // a > 2: later partners by item
  // Device-driven rounds: mL, GL and h from the round state (mL above then
  // bounds the grid only). NULL: the fields above.
  const RoundState *rs;
  uint32_t grid_cap;        // at most this many blocks (grid-stride; 0: one item per thread)
};
cudaError_t launch_gather_large(const GatherLargeArgs &a, cudaStream_t stream);

// The two steps between and after the sorts of an a-tuple round (a > 2).
// rekey: (ka, va)[x] = (key1_stash[j], j) for j = plan->vfinal[x].
// finish: plan->vfinal[y] = gapped position of item j = plan->vfinal[y];
// the other key buffer (kb if the result is in ka, else ka) gets
// sec_stash[j] at y.
struct WideArgs {
  const SortPlan *plan;
  uint32_t m;               // items in the active list (bounds guard)
  uint32_t mL, GL, W;
  const uint64_t *act;
  const uint32_t *gstart;
  const uint32_t *lg, *loff;
  const uint64_t *key1_stash, *sec_stash;
  uint64_t *ka, *kb;
  uint32_t *va;
  Ctrl *ctrl;
};
cudaError_t launch_wide_rekey(const WideArgs &a, cudaStream_t stream);
cudaError_t launch_wide_finish(const WideArgs &a, cudaStream_t stream);

struct RefineArgs {
  const uint64_t *act;      // current active list (g << 32) | i'
  const uint32_t *gstart;   // G + 1 entries
  const uint32_t *gname;
  const uint32_t *ghead;    // head rank of each group
  uint32_t naming;          // NamingRule
  const uint32_t *tfirst;   // tiles + 1 entries
  uint32_t shape;           // index into REFINE_SHAPE
  uint32_t m, G, tiles;
  uint32_t h, W;
  uint32_t mult;            // a: names of i' + h .. i' + (a-1)h are ranked (2, 3, 4)
  const uint32_t *isa;      // read only (updates are deferred)
  uint64_t isa_len;
  uint32_t N;
  uint32_t *sa;             // written with indices local to each text
  const uint32_t *seg_off;  // S + 1 ungapped offsets
  uint32_t S;
  uint64_t *act_out;
  uint32_t *gstart_out, *gname_out, *ghead_out;
  uint64_t *upd;            // (new << 32) | i' for every changed name
  Ctrl *ctrl;               // rc.m_s / rc.g_s / rc.upd reserve the outputs
  // Device-driven rounds: tiles and h from the round state (tiles above
  // then bounds the grid only). NULL: the fields above.
  const RoundState *rs;
  uint32_t grid_cap;        // at most this many blocks, each looping over tiles (0: one per tile)
};
cudaError_t launch_refine(const RefineArgs &a, cudaStream_t stream);

// ISA[i'] = gname[g] for the entries act[*lo, *lo + *count) whose group
// name differs from their parent's (the rename's survivors, or a bucketed
// copy of them); *count <= max_count. Blocks take consecutive chunks in
// launch order.
// translated (host-driven): the entries are (name << 32) | i' of a
// translating bucket pass, all to be written, and *count their number.
// Device-driven rounds (rs): nothing when rs->mL = 0; with rs->bucket_surv
// the entries are the translated bucketed[0, *bucketed_count) instead.
// grid_cap: at most this many blocks (0: one per chunk).
cudaError_t launch_apply_names(const uint64_t *act, const uint32_t *lo, const uint32_t *count,
                               uint32_t max_count, const uint32_t *gname, const uint32_t *gold,
                               uint32_t *isa, uint64_t isa_len, cudaStream_t stream,
                               uint32_t translated = 0, const uint64_t *bucketed = nullptr,
                               const uint32_t *zero = nullptr,
                               const uint32_t *bucketed_count = nullptr,
                               const RoundState *rs = nullptr, uint32_t grid_cap = 0);

// ISA[i'] = new for the min(ctrl->rc.upd, max_upd) queued updates; blocks
// take consecutive chunks in launch order. Device-driven rounds (rs): the
// updates are bucketed[...] when rs->bucket_upd.
cudaError_t launch_scatter_updates(const uint64_t *upd, uint32_t max_upd, uint32_t *isa,
                                   uint64_t isa_len, Ctrl *ctrl, cudaStream_t stream,
                                   const uint64_t *bucketed = nullptr,
                                   const RoundState *rs = nullptr, uint32_t grid_cap = 0);

// ---- device-driven rounds (k_rounds.cu) ------------------------------------
// Look-back epochs one device-driven round may use (its launches take the
// offsets 0 .. ROUND_EPOCHS - 1 from the round state's base).
constexpr uint32_t ROUND_EPOCHS = 16;
struct RoundBeginArgs {
  Ctrl *ctrl;               // ctrl->rs, ctrl->rc, ctrl->rec, ctrl->tile_ctr
  uint32_t *hist;           // MAX_PASSES * 256 digit histograms of the large-group sort
  uint32_t W;               // bits of a partner name
  uint32_t nominal;         // refine window (tiles = ceil(m / nominal))
  uint32_t bucket_min;      // discard threshold of the ISA writes
  uint32_t N;               // characters (h never exceeds it)
  // If-nodes of this round: large-group sort, its rename, bucketing of the
  // queued updates, bucketing of the large groups' ISA entries.
  cudaGraphConditionalHandle if_sort, if_rename, if_bucket_upd, if_bucket_surv;
};
cudaError_t launch_round_begin(const RoundBeginArgs &a, cudaStream_t stream);
// Sets `loop` to 1 while suffixes are active and no error was raised.
cudaError_t launch_round_end(const Ctrl *c, cudaGraphConditionalHandle loop, cudaStream_t stream);

// ---- group order after round 0 (k_reorder.cu) -------------------------------
// keys[g] = the smallest member position of group g, vals[g] = g,
// info[g] = (start, size, name, head rank).
cudaError_t launch_group_minpos(const uint64_t *act, const uint32_t *gstart, const uint32_t *gname,
                                const uint32_t *ghead, uint32_t G, uint64_t *keys, uint32_t *vals,
                                uint4 *info, int num_sms, cudaStream_t stream);
// info_new[x] = info[plan->vfinal[x]], sizes[x] = its size.
cudaError_t launch_group_sizes(const SortPlan *plan, const uint4 *info, uint32_t G,
                               uint4 *info_new, uint32_t *sizes, Ctrl *ctrl, int num_sms,
                               cudaStream_t stream);
// out[i] = in[0] + .. + in[i] (may alias); sums: inclusive_scan_sums_words(m) words.
cudaError_t launch_inclusive_scan(const uint32_t *in, uint32_t *out, uint64_t m, uint32_t *sums,
                                  cudaStream_t stream);
uint64_t inclusive_scan_sums_words(uint64_t m);
struct RegroupArgs {
  const uint4 *info;        // (start, size, name, head rank) of new group x
  const uint64_t *act_in;   // entries in the old order
  const uint32_t *ends;     // inclusive prefix sums of the sizes in the new order
  uint32_t G, m;
  uint64_t *act_out;        // entries (x << 32) | i' in the new order
  uint32_t *gstart_out, *gname_out, *ghead_out;     // G + 1, G, G entries
  Ctrl *ctrl;
};
cudaError_t launch_regroup(const RegroupArgs &a, int num_sms, cudaStream_t stream);

// ---- position bucketing of ISA writes (k_bucket.cu) ------------------------
constexpr uint32_t BUCKET_BLOCKS_MAX = 1024;
struct BucketArgs {
  const uint64_t *in;     // entries (x << 32) | i'
  const uint32_t *lo;     // device word: first entry (NULL: 0)
  const uint32_t *count;  // device word: number of entries
  uint32_t max_count;     // capacity of `in` past *lo and of `out`
  uint32_t shift;         // bucket of an entry: min(i' >> shift, 255)
  uint32_t blocks;        // partition blocks (<= BUCKET_BLOCKS_MAX)
  uint32_t *counts;       // blocks x 256 words: counts, then run starts
  uint64_t *out;          // entries grouped by bucket
  // Translation (the rename's survivors, entries (g << 32) | i'): when
  // gname is set, an entry whose group's name equals its parent's (gold) is
  // dropped and the others are written as (gname[g] << 32) | i', so that
  // the ISA writes need no group lookups; the number written goes to
  // *total_out. Entries come in group order, so these lookups are nearly
  // sequential here and would be random after the partition.
  const uint32_t *gname, *gold;
  uint32_t *total_out;
};
cudaError_t launch_bucket_count(const BucketArgs &a, cudaStream_t stream);
cudaError_t launch_bucket_offsets(const BucketArgs &a, cudaStream_t stream);
cudaError_t launch_bucket_scatter(const BucketArgs &a, cudaStream_t stream);

// ---- output (k_gather.cu) ------------------------------------------------
// isa_out[p] = isa[p + s] - off_s for text s (single text: a copy).
cudaError_t launch_isa_to_local(const uint32_t *isa, uint32_t *isa_out, uint32_t N,
                                const uint32_t *seg_off, uint32_t S, cudaStream_t stream);

}  // namespace gbsa
