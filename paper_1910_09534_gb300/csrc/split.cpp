// split.cpp -- contraction deferral: the two subcircuit gate lists of Sect. 2, with the
// Appendix's EI and E2Q operations written as ordinary gates on fresh wires.
//
// A tensor is simulated as a state over "wires": its side's qubits plus two wires per bridging
// gate, all starting in |0>.  EI on qubit a: a fan-out gate F (first column |00> + |11>) on two
// fresh wires (w1, w2) makes delta(w1, w2); w1 carries qubit a from then on, w2 is the pair's
// a', and a's previous wire, which no later gate touches, is the pair's a.  E2Q on qubit b: F on
// two fresh wires (v1, v2) gives sum_x |x>_v1 |x>_v2; the bridging gate G then acts on (v1, b)
// with v1 in the role of qubit a, so v1 ends as a' = G's output for a, v2 keeps a = G's input,
// and b's wire holds b''.  Both tensors number their pairs in the order of the bridging gates.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace sycsim;

namespace {

// 4x4 fan-out, index b(q0) + 2 b(q1): |00> -> |00> + |11>.  The other columns (never reached
// from fresh wires) complete sqrt(2) times an orthogonal matrix so fused blocks stay well scaled.
void fanout_gate(int w0, int w1, sim_gate &g)
{
    std::memset(&g, 0, sizeof g);
    g.kind = SIM_GATE_U2;
    g.q0 = w0;
    g.q1 = w1;
    static const double m[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, 1, -1, 0}, {1, 0, 0, -1}};
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) g.u[2 * (4 * r + c)] = m[r][c];
}

}  // namespace

extern "C" int sim_split_create(int n_qubits, int n_gates, const sim_gate *gates, const int *side,
                                sim_split_t **out)
{
    if (!out) return fail(nullptr, SIM_E_INVAL, "sim_split_create: NULL out");
    *out = nullptr;
    if (n_qubits < 2 || n_qubits > kMaxQubits || !side || n_gates < 0 || (n_gates > 0 && !gates))
        return fail(nullptr, SIM_E_INVAL, "sim_split_create: bad arguments");
    int n_side[2] = {0, 0}, live[kMaxQubits];
    for (int q = 0; q < n_qubits; ++q) {
        if (side[q] != 0 && side[q] != 1)
            return fail(nullptr, SIM_E_INVAL, "sim_split_create: side[%d] = %d is not 0 or 1", q, side[q]);
        live[q] = n_side[side[q]]++;
    }
    if (n_side[0] == 0 || n_side[1] == 0)
        return fail(nullptr, SIM_E_INVAL, "sim_split_create: both sides need qubits");
    int pairs = 0;
    for (int i = 0; i < n_gates; ++i) {
        const sim_gate &g = gates[i];
        double m[32];
        const int d = gate_matrix(g, m);
        if (d == 0 || g.q0 < 0 || g.q0 >= n_qubits)
            return fail(nullptr, SIM_E_INVAL, "sim_split_create: bad gate %d", i);
        if (d == 4) {
            if (g.q1 < 0 || g.q1 >= n_qubits || g.q1 == g.q0)
                return fail(nullptr, SIM_E_INVAL, "sim_split_create: bad qubits in gate %d", i);
            if (side[g.q0] != side[g.q1]) ++pairs;
        }
    }
    for (int t = 0; t < 2; ++t)
        if (n_side[t] + 2 * pairs > kMaxQubits)
            return fail(nullptr, SIM_E_INVAL, "sim_split_create: tensor %d needs %d wires (limit %d)", t + 1,
                        n_side[t] + 2 * pairs, kMaxQubits);

    sim_split_s *s = new (std::nothrow) sim_split_s;
    if (!s) return fail(nullptr, SIM_E_NOMEM_HOST, "sim_split_create: out of host memory");
    s->n = n_qubits;
    s->n_side[0] = n_side[0];
    s->n_side[1] = n_side[1];
    s->n_pairs = pairs;
    s->side.assign(side, side + n_qubits);
    std::vector<int> pair_ap[2], pair_a[2];  // wires of a'_j, a_j in each tensor
    int j = 0;
    for (int i = 0; i < n_gates; ++i) {
        sim_gate g = gates[i];
        double m[32];
        const bool two = gate_matrix(g, m) == 4;
        if (!two || side[g.q0] == side[g.q1]) {
            const int t = side[g.q0];
            g.q0 = live[g.q0];
            if (two) g.q1 = live[g.q1];
            s->gates[t].push_back(g);
            continue;
        }
        const bool a_is_q0 = side[g.q0] == 0;
        const int a = a_is_q0 ? g.q0 : g.q1, b = a_is_q0 ? g.q1 : g.q0;
        sim_gate f;
        // EI on tensor 1
        const int w1 = n_side[0] + 2 * j, w2 = w1 + 1;
        fanout_gate(w1, w2, f);
        s->gates[0].push_back(f);
        pair_ap[0].push_back(w2);
        pair_a[0].push_back(live[a]);
        live[a] = w1;
        // E2Q on tensor 2
        const int v1 = n_side[1] + 2 * j, v2 = v1 + 1;
        fanout_gate(v1, v2, f);
        s->gates[1].push_back(f);
        if (a_is_q0) {
            g.q0 = v1;
            g.q1 = live[b];
        } else {
            g.q0 = live[b];
            g.q1 = v1;
        }
        s->gates[1].push_back(g);
        pair_ap[1].push_back(v1);
        pair_a[1].push_back(v2);
        ++j;
    }
    for (int t = 0; t < 2; ++t) {
        std::vector<int> &w = s->wire_at[t];
        for (int q = 0; q < n_qubits; ++q)
            if (side[q] == t) w.push_back(live[q]);
        for (int p = 0; p < pairs; ++p) {
            w.push_back(pair_ap[t][p]);
            w.push_back(pair_a[t][p]);
        }
    }
    *out = s;
    return SIM_OK;
}

extern "C" int sim_split_info(const sim_split_t *s, int *n_side, int *n_wires, int *n_pairs, int *n_gates)
{
    if (!s) return fail(nullptr, SIM_E_INVAL, "sim_split_info: NULL split");
    for (int t = 0; t < 2; ++t) {
        if (n_side) n_side[t] = s->n_side[t];
        if (n_wires) n_wires[t] = s->n_side[t] + 2 * s->n_pairs;
        if (n_gates) n_gates[t] = (int)s->gates[t].size();
    }
    if (n_pairs) *n_pairs = s->n_pairs;
    return SIM_OK;
}

extern "C" int sim_split_gates(const sim_split_t *s, int t, sim_gate *out)
{
    if (!s || (t != 0 && t != 1) || !out) return fail(nullptr, SIM_E_INVAL, "sim_split_gates: bad arguments");
    if (!s->gates[t].empty()) std::memcpy(out, s->gates[t].data(), s->gates[t].size() * sizeof(sim_gate));
    return SIM_OK;
}

extern "C" int sim_split_canonical(const sim_split_t *s, int t, int *wire_at)
{
    if (!s || (t != 0 && t != 1) || !wire_at)
        return fail(nullptr, SIM_E_INVAL, "sim_split_canonical: bad arguments");
    for (size_t p = 0; p < s->wire_at[t].size(); ++p) wire_at[p] = s->wire_at[t][p];
    return SIM_OK;
}

extern "C" int sim_split_destroy(sim_split_t *s)
{
    delete s;
    return SIM_OK;
}

struct sim_front_s {
    sim_split_s split;
    sim_t *t[2] = {nullptr, nullptr};
    sim_plan_t *p[2] = {nullptr, nullptr};
    int device = 0;
    int contract_precision = SIM_FP32;
    std::vector<int> lay_for;             // output layout the tensor layouts below were chosen for
    int lay[2][kMaxQubits] = {};          // each tensor's layout (wire -> bit)
};



namespace sycsim {

void front_tensor_layout(const sim_split_s *s, const sim_plan_s *plan, int t, const int *out_bit_of, int *lay, int top)
{
    const int ns = s->n_side[t], nw = (int)s->wire_at[t].size();
    contract_layout(s, out_bit_of, t, lay, nullptr);
    if (ns - top < 5) return;
    int wire_on[kMaxQubits];  // side wire on each of bits 0 .. ns-1 in contract_layout's order
    for (int p = 0; p < ns; ++p) wire_on[lay[s->wire_at[t][p]]] = s->wire_at[t][p];
    const int pool = t == 0 ? 5 : ns - top;  // the low-4 set is drawn from bits 0 .. pool-1
    int cand[kMaxQubits];
    std::copy(lay, lay + nw, cand);
    double best = plan_estimate_ms(plan, lay);
    int c[4] = {0, 1, 2, 3};
    for (;;) {
        // bits 0-3: the chosen four in their order; then the other side wires in order
        int b = 4;
        for (int j = 0; j < ns; ++j) {
            const int *at = std::find(c, c + 4, j);
            cand[wire_on[j]] = at != c + 4 ? (int)(at - c) : b++;
        }
        const double est = plan_estimate_ms(plan, cand);
        if (est < best - 1e-9) {
            best = est;
            std::copy(cand, cand + nw, lay);
        }
        int i = 3;  // next 4-subset of 0 .. pool-1 in lexicographic order
        while (i >= 0 && c[i] == pool - 4 + i) --i;
        if (i < 0) break;
        ++c[i];
        for (int j = i + 1; j < 4; ++j) c[j] = c[j - 1] + 1;
    }
}

}  // namespace sycsim

extern "C" int sim_front_destroy(sim_front_t *f)
{
    if (!f) return fail(nullptr, SIM_E_INVAL, "sim_front_destroy: NULL front");
    for (int t = 0; t < 2; ++t) {
        if (f->p[t]) sim_plan_destroy(f->p[t]);
        if (f->t[t]) sim_destroy(f->t[t]);
    }
    delete f;
    return SIM_OK;
}

extern "C" int sim_front_create(sim_t *out, const sim_split_t *s, const sim_plan_opts *o, sim_front_t **f)
{
    if (!f) return fail(out, SIM_E_INVAL, "sim_front_create: NULL out pointer");
    *f = nullptr;
    if (!out || !s) return fail(out, SIM_E_INVAL, "sim_front_create: NULL argument");
    sim_plan_opts po{};
    po.kmax = 4;
    po.precision = SIM_FP32;
    if (o) po = *o;
    sim_front_s *fr = new (std::nothrow) sim_front_s;
    if (!fr) return fail(out, SIM_E_NOMEM_HOST, "sim_front_create: out of host memory");
    fr->split = *s;
    fr->device = out->device;
    fr->contract_precision = po.precision == SIM_BF16X3 ? SIM_BF16X3
                             : (po.precision == SIM_FP16X3 || po.precision == SIM_FP16X3_TMEM) ? SIM_FP16X3_TMEM
                                                                                                : SIM_FP32;
    for (int t = 0; t < 2; ++t) {
        const int nw = s->n_side[t] + 2 * s->n_pairs;
        int rc = sim_plan_create(nw, (int)s->gates[t].size(), s->gates[t].data(), &po, &fr->p[t]);
        if (rc == SIM_OK) {
            sim_opts so{};
            so.store = SIM_STORE_DEVICE;
            so.device = out->device;
            so.stream = out->stream;
            rc = sim_create(nw, 0, &so, &fr->t[t]);
        }
        if (rc != SIM_OK) {
            const std::string msg = thread_error();
            sim_front_destroy(fr);
            return fail(out, rc, "sim_front_create: tensor %d: %s", t + 1, msg.c_str());
        }
    }
    *f = fr;
    return SIM_OK;
}

extern "C" int sim_front_run_phase(sim_t *out, sim_front_t *f, int set, const sim_plan_t *p)
{
    if (!out || !f) return fail(out, SIM_E_INVAL, "sim_front_run: NULL argument");
    state_written(out);
    if (out->device != f->device) return fail(out, SIM_E_INVAL, "sim_front_run: out is on another device");
    if (out->n != f->split.n)
        return fail(out, SIM_E_INVAL, "sim_front_run: out has %d qubits, the split %d", out->n, f->split.n);
    if (set < 0 || set > 1) return fail(out, SIM_E_INVAL, "sim_front_run: set must be 0 (A) or 1 (B)");
    // into a host store, the contraction writes slices of the sliced set in store_fill_layout's
    // layout; each side's qubits of that set stay on its tensor's top side bits
    int olay[kMaxQubits], top[2] = {0, 0};
    if (out->store == SIM_STORE_HOST) {
        store_fill_layout(out, set, olay);
        for (int i = 0; i < out->s; i++) top[f->split.side[out->set[set][i]]]++;
    } else {
        std::copy(out->bit_of, out->bit_of + out->n, olay);
    }
    if (f->lay_for.size() != (size_t)out->n + 2 || !std::equal(olay, olay + out->n, f->lay_for.begin()) ||
        f->lay_for[out->n] != top[0] || f->lay_for[out->n + 1] != top[1]) {
        for (int t = 0; t < 2; ++t) front_tensor_layout(&f->split, f->p[t], t, olay, f->lay[t], top[t]);
        f->lay_for.assign(olay, olay + out->n);
        f->lay_for.push_back(top[0]);
        f->lay_for.push_back(top[1]);
    }
    for (int t = 0; t < 2; ++t) {
        // relabel the tensor (free: its state is reset next) into a layout the contraction into
        // out reads as it is, so that no run permutes
        const int *lay = f->lay[t];
        for (int w = 0; w < f->t[t]->n; ++w) {
            f->t[t]->bit_of[w] = lay[w];
            f->t[t]->qubit_at[lay[w]] = w;
        }
        const uint64_t before = f->t[t]->launches;
        int rc = sim_reset(f->t[t], 0);
        if (rc == SIM_OK) rc = sim_apply_plan(f->t[t], f->p[t]);
        out->launches += f->t[t]->launches - before;  // the front's kernels count as out's
        if (rc != SIM_OK) return fail(out, rc, "sim_front_run: tensor %d: %s", t + 1, f->t[t]->err.c_str());
    }
    return sim_contract_phase(out, f->t[0], f->t[1], &f->split, f->contract_precision, set, p);
}

extern "C" int sim_front_run(sim_t *out, sim_front_t *f) { return sim_front_run_phase(out, f, 0, nullptr); }

namespace {

// Positions of the (max_pairs + 1)-th .. (max_pairs + 4)-th gates that cross the split (n_gates
// where there are fewer), then the negated imbalance: larger is better, compared in order.
struct SplitScore {
    int pos[4];
    int balance;
    bool operator>(const SplitScore &o) const
    {
        for (int i = 0; i < 4; ++i)
            if (pos[i] != o.pos[i]) return pos[i] > o.pos[i];
        return balance > o.balance;
    }
};

SplitScore split_score(const std::vector<std::pair<int, int>> &two, const std::vector<int> &gate_index,
                       int n_gates, const std::vector<char> &side, int max_pairs, int n)
{
    SplitScore sc{{n_gates, n_gates, n_gates, n_gates}, 0};
    int pairs = 0, k = 0;
    for (size_t i = 0; i < two.size() && k < 4; ++i)
        if (side[two[i].first] != side[two[i].second] && ++pairs > max_pairs) sc.pos[k++] = gate_index[i];
    int a = 0;
    for (int q = 0; q < n; ++q) a += side[q] == 0;
    sc.balance = -std::abs(2 * a - n);
    return sc;
}

}  // namespace

namespace sycsim {

int split_choose(int n_qubits, int n_gates, const sim_gate *gates, int max_pairs, int min_side, int *side,
                 int *n_front, int max_seeds);

}  // namespace sycsim

extern "C" int sim_split_choose(int n_qubits, int n_gates, const sim_gate *gates, int max_pairs, int min_side,
                                int *side, int *n_front)
{
    return split_choose(n_qubits, n_gates, gates, max_pairs, min_side, side, n_front, n_qubits);
}

// The search of sim_split_choose from max_seeds seed qubits spread evenly over 0 .. n-1.
int sycsim::split_choose(int n_qubits, int n_gates, const sim_gate *gates, int max_pairs, int min_side, int *side,
                         int *n_front, int max_seeds)
{
    if (n_qubits < 2 || n_qubits > kMaxQubits || n_gates < 0 || (n_gates > 0 && !gates) || max_pairs < 0 || !side ||
        !n_front)
        return fail(nullptr, SIM_E_INVAL, "sim_split_choose: bad arguments");
    const int n = n_qubits;
    if (min_side <= 0) min_side = 7;
    min_side = std::min(min_side, n / 2);
    const int slack = std::max(1, n / 8);
    const int lo = std::max(min_side, n / 2 - slack), hi = std::min(n - min_side, (n + 1) / 2 + slack);
    // the two-qubit gates in order, and the couplings between qubits
    std::vector<std::pair<int, int>> two;
    std::vector<int> gate_index;
    std::vector<std::vector<int>> adj(n);
    for (int i = 0; i < n_gates; ++i) {
        double m[32];
        const int d = gate_matrix(gates[i], m);
        if (d == 0 || gates[i].q0 < 0 || gates[i].q0 >= n)
            return fail(nullptr, SIM_E_INVAL, "sim_split_choose: bad gate %d", i);
        if (d != 4) continue;
        const int a = gates[i].q0, b = gates[i].q1;
        if (b < 0 || b >= n || a == b) return fail(nullptr, SIM_E_INVAL, "sim_split_choose: bad qubits in gate %d", i);
        two.push_back({a, b});
        gate_index.push_back(i);
        if (std::find(adj[a].begin(), adj[a].end(), b) == adj[a].end()) {
            adj[a].push_back(b);
            adj[b].push_back(a);
        }
    }
    for (auto &v : adj) std::sort(v.begin(), v.end());
    std::vector<char> best_side;
    SplitScore best{};
    bool have = false;
    const int seeds = std::max(1, std::min(max_seeds, n));
    for (int si = 0; si < seeds; ++si) {
        const int seed = (int)((int64_t)si * n / seeds);
        // a half grown breadth-first from the seed over the couplings, topped up in qubit order
        std::vector<char> sd(n, 1);
        std::vector<int> order{seed};
        sd[seed] = 0;
        int cnt = 1;
        for (size_t qi = 0; qi < order.size() && cnt < n / 2; ++qi)
            for (int v : adj[order[qi]])
                if (sd[v] == 1 && cnt < n / 2) {
                    sd[v] = 0;
                    ++cnt;
                    order.push_back(v);
                }
        for (int q = 0; q < n && cnt < n / 2; ++q)
            if (sd[q] == 1) sd[q] = 0, ++cnt;
        SplitScore cur = split_score(two, gate_index, n_gates, sd, max_pairs, n);
        for (int iter = 0; iter < 4 * n; ++iter) {  // best improving move, until none
            SplitScore bm{};
            int ba = -1, bb = -1;
            bool found = false;
            for (int a = 0; a < n; ++a) {  // one qubit to the other side
                const int size0 = cnt + (sd[a] ? 1 : -1);
                if (size0 < lo || size0 > hi) continue;
                sd[a] ^= 1;
                const SplitScore g = split_score(two, gate_index, n_gates, sd, max_pairs, n);
                sd[a] ^= 1;
                if (g > cur && (!found || g > bm)) bm = g, ba = a, bb = -1, found = true;
            }
            for (int a = 0; a < n; ++a) {  // an exchange
                if (sd[a] != 0) continue;
                for (int b = 0; b < n; ++b) {
                    if (sd[b] != 1) continue;
                    sd[a] = 1, sd[b] = 0;
                    const SplitScore g = split_score(two, gate_index, n_gates, sd, max_pairs, n);
                    sd[a] = 0, sd[b] = 1;
                    if (g > cur && (!found || g > bm)) bm = g, ba = a, bb = b, found = true;
                }
            }
            if (!found) break;
            if (bb < 0) cnt += sd[ba] ? 1 : -1;  // a move changes the sizes, an exchange does not
            sd[ba] ^= 1;
            if (bb >= 0) sd[bb] ^= 1;
            cur = bm;
        }
        if (cnt >= lo && cnt <= hi && (!have || cur > best)) {
            best = cur;
            best_side = sd;
            have = true;
        }
    }
    if (!have) return fail(nullptr, SIM_E_INVAL, "sim_split_choose: no split with sides of >= %d qubits", min_side);
    for (int q = 0; q < n; ++q) side[q] = best_side[q];
    *n_front = best.pos[0];
    return SIM_OK;
}
