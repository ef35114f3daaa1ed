// The autotuner's table inside the library: tuned build parameters per
// workload class, consulted by every build whose sa_options leave a knob at
// 0 (automatic).
//
// Key: (batched or single text, bits per character b of the input's
// alphabet, floor(log2 N) of the total length). A build takes the entry of
// its own (batched, b) class whose size bucket is nearest to its own, else
// the built-in defaults. The knobs are the radix tile (keys per thread),
// the refine tile shape (which also sets the small/large group threshold),
// the characters per initial key, and the discard threshold: how many
// pending ISA writes of discarded and renamed suffixes make the build
// bucket them by position first (below it they are written directly).
//
// The table is read once, at the first lookup, from the file named by the
// environment variable GBSA_TUNING_TABLE, else from tuning.txt beside
// libgbsa.so (written by the project's autotuner, autotune.py). Lines:
//   batched bits log2n sort_items refine_shape h0_chars bucket_min
// ('#' starts a comment; a 0 field keeps the built-in default). Entries can
// also be set through sa_tuning_set. Thread-safe.
//
// The paper has no counterpart: this is the runtime's parameter choice for
// the sort and discard steps of Section 2.1.
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/gbsa.h"
#include "launch.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {
namespace {

using Key = std::tuple<uint32_t, uint32_t, uint32_t>;  // (batched, bits, log2n)

std::mutex g_mu;
std::map<Key, sa_tuned> g_table;
bool g_loaded = false;
std::string g_source;  // where the table came from ("" = nowhere)

// Appends the entries of one table file; returns the number read or -1 if
// the file cannot be opened or a line is malformed (nothing is kept then).
int parse_file(const char *path, std::map<Key, sa_tuned> &out) {
  FILE *f = fopen(path, "r");
  if (!f) return -1;
  std::map<Key, sa_tuned> got;
  char line[512];
  int count = 0;
  bool bad = false;
  while (fgets(line, sizeof(line), f)) {
    char *hash = strchr(line, '#');
    if (hash) *hash = 0;
    unsigned batched, bits, log2n, items, shape, h0;
    unsigned long long bmin;
    char extra[2];
    const int k = sscanf(line, "%u %u %u %u %u %u %llu %1s", &batched, &bits, &log2n, &items,
                         &shape, &h0, &bmin, extra);
    if (k <= 0) continue;  // blank or comment
    if (k != 7 || batched > 1 || bits < 1 || bits > 8 || log2n > 31 || bmin > 0xFFFFFFFFull) {
      bad = true;
      break;
    }
    sa_tuned t{};
    t.sort_items = items;
    t.refine_shape = shape;
    t.h0_chars = h0;
    t.bucket_min = (uint32_t)bmin;
    got[Key{batched, bits, log2n}] = t;
    ++count;
  }
  fclose(f);
  if (bad) return -1;
  for (auto &kv : got) out[kv.first] = kv.second;
  return count;
}

std::string default_path() {
  const char *env = getenv("GBSA_TUNING_TABLE");
  if (env && *env) return env;
  Dl_info info{};
  if (dladdr(reinterpret_cast<void *>(&sa_tuning_load), &info) && info.dli_fname) {
    std::string p(info.dli_fname);
    const size_t slash = p.rfind('/');
    return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/tuning.txt";
  }
  return "tuning.txt";
}

void load_default_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string p = default_path();
  if (parse_file(p.c_str(), g_table) >= 0) g_source = p;
}

}  // namespace

void tuned_params(bool batched, uint32_t bits, uint64_t n, sa_tuned *out) {
  *out = sa_tuned{};
  uint32_t log2n = 0;
  while (log2n < 63 && (n >> (log2n + 1)) != 0) ++log2n;
  std::lock_guard<std::mutex> g(g_mu);
  load_default_locked();
  const sa_tuned *best = nullptr;
  uint32_t dist = 0;
  for (auto &kv : g_table) {
    if (std::get<0>(kv.first) != (batched ? 1u : 0u) || std::get<1>(kv.first) != bits) continue;
    const uint32_t b = std::get<2>(kv.first);
    const uint32_t d = b > log2n ? b - log2n : log2n - b;
    if (!best || d < dist) {
      best = &kv.second;
      dist = d;
    }
  }
  if (best) *out = *best;
}

}  // namespace gbsa

using namespace gbsa;

GBSA_API sa_status sa_tuning_set(uint32_t batched, uint32_t bits_per_char, uint32_t log2_n,
                                 const sa_tuned *params) {
  if (batched > 1 || bits_per_char < 1 || bits_per_char > 8 || log2_n > 31)
    return SA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  load_default_locked();
  const Key k{batched, bits_per_char, log2_n};
  if (params)
    g_table[k] = *params;
  else
    g_table.erase(k);
  return SA_OK;
}

GBSA_API sa_status sa_tuning_load(const char *path) {
  std::lock_guard<std::mutex> g(g_mu);
  g_loaded = true;  // an explicit table replaces the default file
  if (!path) {
    g_table.clear();
    g_source.clear();
    return SA_OK;
  }
  std::map<Key, sa_tuned> t;
  if (parse_file(path, t) < 0) return SA_ERR_INVALID_ARG;
  g_table.swap(t);
  g_source = path;
  return SA_OK;
}

GBSA_API uint32_t sa_tuning_lookup(uint32_t batched, uint32_t bits_per_char, uint64_t n,
                                   sa_tuned *out) {
  if (!out) return 0;
  tuned_params(batched != 0, bits_per_char, n, out);
  std::lock_guard<std::mutex> g(g_mu);
  return (uint32_t)g_table.size();
}
