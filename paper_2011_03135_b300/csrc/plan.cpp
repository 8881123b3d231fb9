// Pattern planner (host). For an explicit pattern given by its adjacency
// matrix it derives what the paper's high-level engine derives before a
// search (Section 4.3 "High Level Optimizations" and appendix "Symmetry
// Breaking (Partial Order)", "Orientation (Total Order)", "Pattern-Guided
// Search (Matching Order)"):
//   - |Aut(P)| by testing all k! vertex permutations (k <= 8);
//   - symmetry-breaking constraints id(f(a)) < id(f(b)) from the stabiliser
//     chain of Aut(P): fix pattern vertices in index order; every other vertex
//     in the current orbit of the fixed vertex must map to a larger id; then
//     restrict the group to the stabiliser (Grochow & Kellis, RECOMB 2007).
//     The constraints leave exactly k!/|Aut(P)| vertex orders, one per
//     distinct subgraph;
//   - a greedy matching order: start from the edge that carries the most
//     constraints, then repeatedly add the connected vertex that brings the
//     most constraints, then the most edges, into the matched set (ties: the
//     lower index) -- for the diamond this matches the triangle first with
//     the constraint between the two degree-3 vertices, the order the paper
//     selects;
//   - degree filter thresholds (each pattern vertex's degree, Section 4.3 DF);
//   - the execution strategy: the orientation for cliques (the paper enables
//     it exactly when |E| = |V|(|V|-1)/2), local counting for the other 3- and
//     4-vertex patterns (Section 5), pattern-oblivious enumeration with
//     connectivity codes for the other 5-vertex patterns (Section 4.2).
#include <algorithm>
#include <cstring>
#include <vector>

#include "gpm_internal.h"

namespace {

using Perm = std::vector<uint32_t>;

bool is_automorphism(const gpm_pattern &p, const Perm &s) {
  const uint32_t k = p.k;
  for (uint32_t i = 0; i < k; ++i)
    for (uint32_t j = 0; j < k; ++j)
      if ((p.adj[s[i] * k + s[j]] != 0) != (p.adj[i * k + j] != 0)) return false;
  return true;
}

// all permutations s of 0..k-1 with pat(s(i), s(j)) == tmpl(i, j)
std::vector<Perm> isomorphisms(uint32_t k, const uint8_t *tmpl, const uint8_t *pat) {
  std::vector<Perm> out;
  Perm s(k);
  for (uint32_t i = 0; i < k; ++i) s[i] = i;
  do {
    bool ok = true;
    for (uint32_t i = 0; i < k && ok; ++i)
      for (uint32_t j = 0; j < k; ++j)
        if ((pat[s[i] * k + s[j]] != 0) != (tmpl[i * k + j] != 0)) {
          ok = false;
          break;
        }
    if (ok) out.push_back(s);
  } while (std::next_permutation(s.begin(), s.end()));
  return out;
}

bool connected(const gpm_pattern &p) {
  const uint32_t k = p.k;
  uint32_t seen = 1u, frontier = 1u;
  while (frontier) {
    uint32_t next = 0;
    for (uint32_t v = 0; v < k; ++v)
      if (frontier >> v & 1u)
        for (uint32_t w = 0; w < k; ++w)
          if (p.adj[v * k + w] && !(seen >> w & 1u)) next |= 1u << w;
    seen |= next;
    frontier = next;
  }
  return seen == (k == 32 ? 0xffffffffu : ((1u << k) - 1u));
}

void set_template(uint8_t *a, uint32_t k, std::initializer_list<std::pair<int, int>> edges) {
  std::memset(a, 0, k * k);
  for (auto e : edges) a[e.first * k + e.second] = a[e.second * k + e.first] = 1;
}

}  // namespace

int gpm_plan_pattern(gpm_pattern *p) {
  const uint32_t k = p->k;
  if (k < 1) return gpm_fail(GPM_E_INVALID_ARG, "pattern needs at least one vertex");
  if (k > 8) return gpm_fail(GPM_E_K_TOO_LARGE, "pattern has more than 8 vertices");
  uint32_t deg[8] = {0};
  uint32_t edges = 0;
  for (uint32_t i = 0; i < k; ++i) {
    if (p->adj[i * k + i]) return gpm_fail(GPM_E_INVALID_ARG, "pattern adjacency has a self-loop");
    for (uint32_t j = 0; j < k; ++j) {
      if (p->adj[i * k + j] > 1) return gpm_fail(GPM_E_INVALID_ARG, "pattern adjacency entries must be 0 or 1");
      if ((p->adj[i * k + j] != 0) != (p->adj[j * k + i] != 0))
        return gpm_fail(GPM_E_INVALID_ARG, "pattern adjacency is not symmetric");
      if (p->adj[i * k + j]) {
        deg[i]++;
        if (j > i) ++edges;
      }
    }
  }
  if (!connected(*p)) return gpm_fail(GPM_E_DISCONNECTED_PATTERN, "pattern is not connected");

  gpm_pattern_info_t &info = p->info;
  std::memset(&info, 0, sizeof(info));
  info.k = k;
  info.n_edges = edges;
  info.induced = p->induced ? 1u : 0u;
  info.is_clique = (edges == k * (k - 1) / 2) ? 1u : 0u;
  info.motif_index = UINT32_MAX;
  for (uint32_t i = 0; i < k; ++i) info.min_degree[i] = deg[i];

  // automorphisms
  std::vector<Perm> group;
  {
    Perm s(k);
    for (uint32_t i = 0; i < k; ++i) s[i] = i;
    do {
      if (is_automorphism(*p, s)) group.push_back(s);
    } while (std::next_permutation(s.begin(), s.end()));
  }
  info.automorphisms = group.size();

  // symmetry breaking from the stabiliser chain
  std::vector<std::pair<uint32_t, uint32_t>> sb;
  for (uint32_t v = 0; v < k && group.size() > 1; ++v) {
    bool in_orbit[8] = {false};
    for (const Perm &s : group) in_orbit[s[v]] = true;
    for (uint32_t u = 0; u < k; ++u)
      if (u != v && in_orbit[u]) sb.emplace_back(v, u);
    std::vector<Perm> stab;
    for (const Perm &s : group)
      if (s[v] == v) stab.push_back(s);
    group.swap(stab);
  }
  info.n_sb_pairs = (uint32_t)sb.size();
  for (size_t i = 0; i < sb.size(); ++i) {
    info.sb_pairs[2 * i] = sb[i].first;
    info.sb_pairs[2 * i + 1] = sb[i].second;
  }

  // greedy matching order
  auto n_cons = [&](uint32_t set) {
    uint32_t c = 0;
    for (auto &pr : sb) c += ((set >> pr.first) & 1u) && ((set >> pr.second) & 1u);
    return c;
  };
  auto n_edges_in = [&](uint32_t set) {
    uint32_t c = 0;
    for (uint32_t i = 0; i < k; ++i)
      for (uint32_t j = i + 1; j < k; ++j) c += ((set >> i) & 1u) && ((set >> j) & 1u) && p->adj[i * k + j];
    return c;
  };
  uint32_t order_len = 0, chosen = 0;
  if (k == 1) {
    info.matching_order[order_len++] = 0;
  } else {
    int best_a = -1, best_b = -1;
    uint32_t best_c = 0;
    for (uint32_t a = 0; a < k; ++a)
      for (uint32_t b = a + 1; b < k; ++b)
        if (p->adj[a * k + b]) {
          uint32_t c = n_cons((1u << a) | (1u << b));
          if (best_a < 0 || c > best_c) {
            best_a = (int)a;
            best_b = (int)b;
            best_c = c;
          }
        }
    info.matching_order[order_len++] = (uint32_t)best_a;
    info.matching_order[order_len++] = (uint32_t)best_b;
    chosen = (1u << best_a) | (1u << best_b);
    while (order_len < k) {
      int best = -1;
      uint32_t bc = 0, be = 0;
      for (uint32_t v = 0; v < k; ++v) {
        if (chosen >> v & 1u) continue;
        bool adjacent = false;
        for (uint32_t w = 0; w < k; ++w) adjacent |= ((chosen >> w) & 1u) && p->adj[v * k + w];
        if (!adjacent) continue;
        const uint32_t c = n_cons(chosen | (1u << v)), e = n_edges_in(chosen | (1u << v));
        if (best < 0 || c > bc || (c == bc && e > be)) {
          best = (int)v;
          bc = c;
          be = e;
        }
      }
      info.matching_order[order_len++] = (uint32_t)best;
      chosen |= 1u << best;
    }
  }

  // class and strategy
  uint32_t ds[8];
  std::memcpy(ds, deg, sizeof(ds));
  std::sort(ds, ds + k);
  if (k == 1) p->cls = PC_VERTEX;
  else if (k == 2) p->cls = PC_EDGE;
  else if (info.is_clique) p->cls = PC_CLIQUE;
  else if (k == 3) p->cls = PC_WEDGE;
  else if (k == 4 && edges == 3 && ds[3] == 3) p->cls = PC_STAR3;
  else if (k == 4 && edges == 3) p->cls = PC_PATH4;
  else if (k == 4 && edges == 4 && ds[3] == 3) p->cls = PC_TAILED;
  else if (k == 4 && edges == 4) p->cls = PC_CYCLE4;
  else if (k == 4 && edges == 5) p->cls = PC_DIAMOND;
  else p->cls = PC_OTHER;
  switch (p->cls) {
    case PC_VERTEX:
    case PC_EDGE: info.strategy = GPM_STRATEGY_EDGE; break;
    case PC_CLIQUE: info.strategy = GPM_STRATEGY_CLIQUE_DAG; break;
    case PC_OTHER: info.strategy = (k == 5) ? GPM_STRATEGY_ENUMERATE : GPM_STRATEGY_GUIDED; break;
    default: info.strategy = GPM_STRATEGY_LOCAL_COUNT; break;
  }
  if (k == 3) info.motif_index = (p->cls == PC_WEDGE) ? 0u : 1u;
  if (k == 5) info.motif_index = (uint32_t)gpm_enum_class_of(*p);
  if (k == 4) {
    switch (p->cls) {
      case PC_STAR3: info.motif_index = 0; break;
      case PC_PATH4: info.motif_index = 1; break;
      case PC_TAILED: info.motif_index = 2; break;
      case PC_CYCLE4: info.motif_index = 3; break;
      case PC_DIAMOND: info.motif_index = 4; break;
      case PC_CLIQUE: info.motif_index = 5; break;
      default: break;
    }
  }

  // template -> pattern isomorphism for listing, chosen so that the
  // template's canonical constraints map onto this pattern's constraints
  for (uint32_t i = 0; i < 8; ++i) p->tmpl_to_pat[i] = i;
  if (p->cls == PC_DIAMOND || p->cls == PC_CYCLE4) {
    uint8_t tmpl[16];
    std::vector<std::pair<uint32_t, uint32_t>> tsb;
    if (p->cls == PC_DIAMOND) {
      set_template(tmpl, 4, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}});
      tsb = {{0, 1}, {2, 3}};
    } else {
      set_template(tmpl, 4, {{0, 2}, {2, 1}, {1, 3}, {3, 0}});
      tsb = {{0, 1}, {0, 2}, {0, 3}, {2, 3}};
    }
    std::vector<std::pair<uint32_t, uint32_t>> want = sb;
    std::sort(want.begin(), want.end());
    bool found = false;
    for (const Perm &s : isomorphisms(4, tmpl, p->adj)) {
      std::vector<std::pair<uint32_t, uint32_t>> mapped;
      for (auto &pr : tsb) mapped.emplace_back(s[pr.first], s[pr.second]);
      std::sort(mapped.begin(), mapped.end());
      if (mapped == want) {
        for (uint32_t i = 0; i < 4; ++i) p->tmpl_to_pat[i] = s[i];
        found = true;
        break;
      }
    }
    if (!found) return gpm_fail(GPM_E_INVALID_ARG, "internal: no template isomorphism matches the constraints");
  }
  return GPM_OK;
}
