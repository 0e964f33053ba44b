// DAG-based gate fusion: Section 5.1 (DAG construction, Eq. 8) and Section 5.2
// (Algorithm 2, U_fused = U_v . U_u of Eq. 9).  Host code; matrix products in FP64.
//
// DAG: scanning gates in order with a "last gate on each qubit" map, an edge (u, v) is
// added for every qubit of v whose last gate is u (|E| <= sum_v |q(v)|).
//
// Sweeps: until a sweep fuses nothing, take the vertices in topological order (Kahn's
// algorithm, smallest vertex id first); for each surviving vertex v try its
// predecessors u -- narrowest union |q(u) U q(v)| first, ties by ascending id (the
// paper leaves the order open; narrow fused gates leave room for later contractions)
// -- and fuse the first u with
//   |q(u) U q(v)| <= max_k   and   no directed path u -> ... -> v other than (u, v),
// i.e. the contraction keeps the graph acyclic, which is how Algorithm 2's "u is the
// sole predecessor of v on the shared qubits" is read here (it also excludes detours
// through other qubits).  u absorbs v: U_u <- E(U_v) . E(U_u) on the sorted union of
// their qubits (E = embedding with identities), v's in- and out-edges move to u, and u
// keeps its id.  The final schedule lists the survivors in the same topological order.
//
// Commutation-aware variant (the paper's fusion does no commutativity analysis and
// names it as future work, Sections 10-11): two gates commute when both are diagonal in
// every qubit they share (neither changes that qubit's bit).  Per qubit, a gate that is
// not diagonal on it depends on every gate on it since the previous such gate, a gate
// diagonal on it only on that previous gate; vertices with no path between them then
// commute.  The sweep also tries, after v's predecessors, the vertices that share a
// qubit with v, are placed before v and are not its predecessors (ascending id), and
// contracts one with no path to v (either product order is the same operator).
#include <algorithm>
#include <queue>
#include <set>

#include "sv_internal.h"

namespace svi {
namespace {

struct Node {
    bool alive = true;
    Gate g;
    std::set<int> preds, succs;   // ordered: predecessors are tried in ascending id
};

// Matrix of gate g (sorted targets) embedded on the sorted qubit set qs (size m):
// g's matrix on its own positions, the identity on the others.
std::vector<cplx> embed(const Gate &g, const uint32_t *qs, uint32_t m) {
    int pos[SV_MAX_K];
    uint32_t amask = 0;
    for (uint32_t j = 0; j < g.k; ++j) {
        uint32_t p = 0;
        while (qs[p] != g.t[j]) ++p;
        pos[j] = (int)p;
        amask |= 1u << p;
    }
    const int d = 1 << m, dg = 1 << g.k;
    int off[1 << SV_MAX_K];
    for (int a = 0; a < dg; ++a) {
        int r = 0;
        for (uint32_t j = 0; j < g.k; ++j) r |= ((a >> j) & 1) << pos[j];
        off[a] = r;
    }
    std::vector<cplx> e((size_t)d * d, cplx(0.0, 0.0));
    for (int e0 = 0; e0 < d; ++e0) {
        if (e0 & amask) continue;                       // the other qubits' values
        for (int ra = 0; ra < dg; ++ra)
            for (int ca = 0; ca < dg; ++ca)
                e[(size_t)(e0 | off[ra]) * d + (e0 | off[ca])] = g.u[(size_t)ra * dg + ca];
    }
    return e;
}

// Positions of g's targets within the sorted set qs, as a bit mask and per target.
static uint32_t target_positions(const Gate &g, const uint32_t *qs, int *pos) {
    uint32_t mask = 0;
    for (uint32_t j = 0; j < g.k; ++j) {
        uint32_t p = 0;
        while (qs[p] != g.t[j]) ++p;
        pos[j] = (int)p;
        mask |= 1u << p;
    }
    return mask;
}

// Spread the bits of a (bit j of a -> bit pos[j]).
static inline int deposit(int a, const int *pos, uint32_t k) {
    int r = 0;
    for (uint32_t j = 0; j < k; ++j) r |= ((a >> j) & 1) << pos[j];
    return r;
}

// Eq. 9: U_fused = U_v . U_u on the sorted qubit set qs (size m), u applied first.  E(U_u)
// is U_u itself when u already acts on all of qs (the common case: u absorbs a narrower
// v); U_v is applied to each column in place of the dense product with E(U_v), entry by
// entry in the same order (nonzero terms of row r, ascending column index).
Gate fused_product(const Gate &gu, const Gate &gv, const uint32_t *qs, uint32_t m) {
    const int d = 1 << m;
    const std::vector<cplx> eu = gu.k == m ? gu.u : embed(gu, qs, m);
    int pv[SV_MAX_K];
    const uint32_t vmask = target_positions(gv, qs, pv);
    const int dv = 1 << gv.k;
    int off[1 << SV_MAX_K];
    for (int a = 0; a < dv; ++a) off[a] = deposit(a, pv, gv.k);
    Gate f;
    f.k = m;
    for (uint32_t j = 0; j < m; ++j) f.t[j] = qs[j];
    f.u.assign((size_t)d * d, cplx(0.0, 0.0));
    for (int r0 = 0; r0 < d; ++r0) {
        if (r0 & vmask) continue;                       // base rows: v's bits clear
        for (int b = 0; b < dv; ++b) {
            cplx *frow = &f.u[(size_t)(r0 | off[b]) * d];
            for (int a = 0; a < dv; ++a) {
                const cplx w = gv.u[(size_t)b * dv + a];
                if (w == cplx(0.0, 0.0)) continue;
                const cplx *urow = &eu[(size_t)(r0 | off[a]) * d];
                for (int c = 0; c < d; ++c) frow[c] += w * urow[c];
            }
        }
    }
    return f;
}

class Dag {
  public:
    Dag(const std::vector<Gate> &gates, uint32_t n, bool commute)
        : nodes_(gates.size()), seen_(gates.size(), 0), pos_(gates.size(), 0), on_qubit_(n) {
        std::vector<int> last(n, -1);
        std::vector<std::vector<int>> diag_since(commute ? n : 0);
        for (size_t i = 0; i < gates.size(); ++i) {
            nodes_[i].g = gates[i];
            const uint32_t dmask = commute ? diagonal_mask(gates[i]) : 0u;
            for (uint32_t j = 0; j < gates[i].k; ++j) {
                const uint32_t q = gates[i].t[j];
                on_qubit_[q].insert((int)i);
                if (!commute) {
                    if (last[q] >= 0) edge(last[q], (int)i);
                    last[q] = (int)i;
                } else if ((dmask >> j) & 1u) {
                    if (last[q] >= 0) edge(last[q], (int)i);
                    diag_since[q].push_back((int)i);
                } else {
                    for (int w : diag_since[q]) edge(w, (int)i);
                    if (last[q] >= 0) edge(last[q], (int)i);
                    diag_since[q].clear();
                    last[q] = (int)i;
                }
            }
        }
    }

    void edge(int u, int v) {
        nodes_[v].preds.insert(u);
        nodes_[u].succs.insert(v);
    }

    // Alive vertices that share a qubit with v, are placed before it in the sweep's
    // order and are not its predecessors, in ascending id.
    std::vector<int> siblings(int v) const {
        std::set<int> out;
        const Node &V = nodes_[v];
        for (uint32_t j = 0; j < V.g.k; ++j)
            for (int w : on_qubit_[V.g.t[j]])
                if (w != v && pos_[w] < pos_[v] && !V.preds.count(w)) out.insert(w);
        return std::vector<int>(out.begin(), out.end());
    }

    std::vector<int> topo_order() const {
        std::vector<int> indeg(nodes_.size(), 0);
        std::priority_queue<int, std::vector<int>, std::greater<int>> ready;
        for (size_t v = 0; v < nodes_.size(); ++v) {
            if (!nodes_[v].alive) continue;
            indeg[v] = (int)nodes_[v].preds.size();
            if (indeg[v] == 0) ready.push((int)v);
        }
        std::vector<int> out;
        while (!ready.empty()) {
            const int v = ready.top();
            ready.pop();
            out.push_back(v);
            for (int w : nodes_[v].succs)
                if (--indeg[w] == 0) ready.push(w);
        }
        return out;
    }

    // Is there a path u -> ... -> v other than the edge (u, v)?  pos_ is the position of
    // each vertex in the topological order the current sweep started from.  During the
    // sweep a contraction keeps the absorbing vertex u at its (earlier) position and only
    // adds edges into it from vertices placed before v, so a vertex placed after v still
    // reaches only vertices placed after v: the search never needs to enter one.
    bool other_path(int u, int v) {
        ++stamp_;
        const int pv = pos_[v];
        stack_.clear();
        for (int w : nodes_[u].succs)
            if (w != v && pos_[w] < pv) { stack_.push_back(w); seen_[w] = stamp_; }
        while (!stack_.empty()) {
            const int w = stack_.back();
            stack_.pop_back();
            for (int x : nodes_[w].succs) {
                if (x == v) return true;
                if (seen_[x] != stamp_ && pos_[x] < pv) { seen_[x] = stamp_; stack_.push_back(x); }
            }
        }
        return false;
    }

    void set_positions(const std::vector<int> &order) {
        for (size_t i = 0; i < order.size(); ++i) pos_[order[i]] = (int)i;
    }

    static uint32_t union_qubits(const Gate &a, const Gate &b, uint32_t *qs) {
        uint32_t m = 0;
        uint32_t i = 0, j = 0;
        while (i < a.k || j < b.k) {
            uint32_t x;
            if (j >= b.k || (i < a.k && a.t[i] < b.t[j])) x = a.t[i++];
            else if (i >= a.k || b.t[j] < a.t[i]) x = b.t[j++];
            else { x = a.t[i]; ++i; ++j; }
            if (m < 2 * SV_MAX_K) qs[m] = x;
            ++m;
        }
        return m;
    }

    void contract(int u, int v, const uint32_t *qs, uint32_t m) {
        Node &U = nodes_[u], &V = nodes_[v];
        for (uint32_t j = 0; j < V.g.k; ++j) on_qubit_[V.g.t[j]].erase(v);
        for (uint32_t j = 0; j < m; ++j) on_qubit_[qs[j]].insert(u);
        U.g = fused_product(U.g, V.g, qs, m);
        for (int w : V.preds)
            if (w != u) {
                nodes_[w].succs.erase(v);
                nodes_[w].succs.insert(u);
                U.preds.insert(w);
            }
        for (int w : V.succs) {
            nodes_[w].preds.erase(v);
            nodes_[w].preds.insert(u);
            U.succs.insert(w);
        }
        U.succs.erase(v);
        V.alive = false;
        V.preds.clear();
        V.succs.clear();
        V.g.u.clear();
    }

    std::vector<Node> nodes_;
    std::vector<uint32_t> seen_;
    std::vector<int> pos_, stack_;
    std::vector<std::set<int>> on_qubit_;   // alive vertices acting on each qubit
    uint32_t stamp_ = 0;
};

}  // namespace

uint32_t diagonal_mask(const Gate &g) {
    const uint32_t d = 1u << g.k;
    uint32_t mask = 0;
    for (uint32_t j = 0; j < g.k; ++j) {
        bool diag = true;
        for (uint32_t r = 0; r < d && diag; ++r)
            for (uint32_t c = 0; c < d; ++c)
                if (((r ^ c) >> j) & 1u && g.u[(size_t)r * d + c] != cplx(0.0, 0.0)) {
                    diag = false;
                    break;
                }
        if (diag) mask |= 1u << j;
    }
    return mask;
}

std::vector<Gate> fuse_gates(const std::vector<Gate> &in, uint32_t n, uint32_t max_k, FusePlan *plan,
                             bool commute) {
    Dag dag(in, n, commute);
    if (plan) plan->contractions.clear();
    bool changed = max_k > 0;
    while (changed) {
        changed = false;
        const std::vector<int> order = dag.topo_order();
        dag.set_positions(order);
        for (int v : order) {
            if (!dag.nodes_[v].alive) continue;
            // candidates: predecessors, then (commute) siblings, each group by (width, id)
            auto by_width = [&](std::vector<int> &c) {
                std::vector<std::pair<uint32_t, int>> w;
                w.reserve(c.size());
                for (int u : c) {
                    uint32_t qs[2 * SV_MAX_K];
                    w.emplace_back(Dag::union_qubits(dag.nodes_[u].g, dag.nodes_[v].g, qs), u);
                }
                std::sort(w.begin(), w.end());
                for (size_t i = 0; i < c.size(); ++i) c[i] = w[i].second;
            };
            std::vector<int> cands(dag.nodes_[v].preds.begin(), dag.nodes_[v].preds.end());
            by_width(cands);
            if (commute) {
                std::vector<int> sib = dag.siblings(v);
                by_width(sib);
                cands.insert(cands.end(), sib.begin(), sib.end());
            }
            for (int u : cands) {
                uint32_t qs[2 * SV_MAX_K];
                const uint32_t m = Dag::union_qubits(dag.nodes_[u].g, dag.nodes_[v].g, qs);
                if (m > max_k) continue;
                if (dag.other_path(u, v)) continue;
                dag.contract(u, v, qs, m);
                if (plan) plan->contractions.emplace_back(u, v);
                changed = true;
                break;
            }
        }
    }
    std::vector<Gate> out;
    const std::vector<int> order = dag.topo_order();
    if (plan) plan->order = order;
    for (int v : order) out.push_back(dag.nodes_[v].g);
    return out;
}

// g widened to m qubits: U (x) I on extra qubits, the smallest non-targets at or above
// bit 5 (below it only if the state is too small), so that the kernels' rows stay
// contiguous in shared memory.
Gate widen_gate(const Gate &g, uint32_t n, uint32_t m) {
    bool used[64] = {false};
    for (uint32_t j = 0; j < g.k; ++j) used[g.t[j]] = true;
    uint32_t k = g.k;
    for (uint32_t q = 5; q < n && k < m; ++q)
        if (!used[q]) { used[q] = true; ++k; }
    for (uint32_t q = 0; q < n && k < m; ++q)
        if (!used[q]) { used[q] = true; ++k; }
    uint32_t qs[SV_MAX_K];
    uint32_t i = 0;
    for (uint32_t q = 0; q < n && i < m; ++q)
        if (used[q]) qs[i++] = q;
    Gate w;
    w.k = m;
    for (uint32_t j = 0; j < m; ++j) w.t[j] = qs[j];
    w.u = embed(g, qs, m);
    return w;
}

// g as an m-qubit gate U (x) I on the sorted qubit set qs (which contains g's targets).
Gate widen_gate_on(const Gate &g, const uint32_t *qs, uint32_t m) {
    Gate w;
    w.k = m;
    for (uint32_t j = 0; j < m; ++j) w.t[j] = qs[j];
    w.u = embed(g, qs, m);
    return w;
}

// Replay a recorded plan on gates with the same qubit sets: Algorithm 2's decisions
// depend only on the qubits, so this yields the schedule fuse_gates would produce, with
// the same products computed in the same order.
std::vector<Gate> replay_fusion(std::vector<Gate> nodes, const FusePlan &plan) {
    for (const auto &uv : plan.contractions) {
        Gate &gu = nodes[uv.first];
        const Gate &gv = nodes[uv.second];
        uint32_t qs[2 * SV_MAX_K];
        const uint32_t m = Dag::union_qubits(gu, gv, qs);
        gu = fused_product(gu, gv, qs, m);
    }
    std::vector<Gate> out;
    out.reserve(plan.order.size());
    for (int v : plan.order) out.push_back(std::move(nodes[v]));
    return out;
}

}  // namespace svi
