// Process-wide table of tuned kernel shapes, keyed by device and problem class, and
// the C-ABI calls that show and clear it.  The entries are written by the kernels'
// host code when a call asks for autotuning (fk_opts.autotune) and the class has no
// entry yet; later calls of the class use the stored shape whether or not they ask.
#include "fk_internal.cuh"

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace fk {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // device, kind, a, b, c, d

struct Entry {
  BinCfg cfg;
  int ival = 0;
  std::string log;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;

Key make_key(const TuneKey& k) {
  int dev = 0;
  cudaGetDevice(&dev);
  return Key{dev, k.kind, k.a, k.b, k.c, k.d};
}

}  // namespace

bool tune_lookup(const TuneKey& k, BinCfg* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(make_key(k));
  if (it == g_table.end()) return false;
  *out = it->second.cfg;
  return true;
}

void tune_store(const TuneKey& k, const BinCfg& v, const std::string& log) {
  std::lock_guard<std::mutex> lock(g_mu);
  Entry& e = g_table[make_key(k)];
  e.cfg = v;
  e.log = log;
}

bool tune_lookup_int(const TuneKey& k, int* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(make_key(k));
  if (it == g_table.end()) return false;
  *out = it->second.ival;
  return true;
}

void tune_store_int(const TuneKey& k, int v, const std::string& log) {
  std::lock_guard<std::mutex> lock(g_mu);
  Entry& e = g_table[make_key(k)];
  e.ival = v;
  e.log = log;
}

}  // namespace fk

using namespace fk;

extern "C" size_t fk_autotune_table(char* buf, size_t cap) {
  std::string out;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto& kv : g_table) {
      const Key& k = kv.first;
      const char* kind = std::get<1>(k) == TUNE_SPREAD2D ? "spread2d"
                         : std::get<1>(k) == TUNE_SPREAD1D ? "spread1d"
                                                            : "cg2d";
      char head[128];
      snprintf(head, sizeof(head), "dev%d %s class(%d,%d,%d,%d): ", std::get<0>(k), kind, std::get<2>(k),
               std::get<3>(k), std::get<4>(k), std::get<5>(k));
      out += head;
      out += kv.second.log;
      out += "\n";
    }
  }
  if (buf && cap > 0) {
    const size_t n = std::min(cap - 1, out.size());
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return out.size() + 1;
}

extern "C" void fk_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
}
