// Process-wide cache of the launch shapes picked by ising_autotune and
// ising_batch_autotune.
#include <map>
#include <mutex>
#include <tuple>

#include "ising_host.h"

namespace isg {

namespace {
std::mutex g_mu;
std::map<TuneKey, int> g_cache;
}  // namespace

bool TuneKey::operator<(const TuneKey& o) const {
  return std::tie(Lx, Ly, Lz, y_mode, x_pbc, exact, m_class) <
         std::tie(o.Lx, o.Ly, o.Lz, o.y_mode, o.x_pbc, o.exact, o.m_class);
}

TuneKey tune_key(const FilmDesc& d, uint32_t measure_every) {
  // records every 1, 2, ... 15 sweeps are told apart; rarer ones cost alike
  const uint32_t m = measure_every == 0 ? 0u : (measure_every < 16 ? measure_every : 16u);
  return TuneKey{d.Lx, d.Ly, d.Lz, d.y_mode, d.x_pbc, d.has_never ? 1u : 0u, m};
}

bool tune_lookup(const TuneKey& k, int* shape) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_cache.find(k);
  if (it == g_cache.end()) return false;
  *shape = it->second;
  return true;
}

void tune_store(const TuneKey& k, int shape) {
  std::lock_guard<std::mutex> g(g_mu);
  g_cache[k] = shape;
}

}  // namespace isg
