// plan.cpp -- gate aggregation planner and FP64 block composition (Sect. 5: gates are
// aggregated into k-qubit kernels, k <= k_max, each a 2^k x 2^k unitary; Appendix A's
// "new cache" lines list such qubit groups and the gates that follow belong to them).
//
// First every single-qubit gate is folded into a neighbouring two-qubit gate (Sect. 3), giving
// "units" of at most two qubits.  Then blocks are formed one at a time from the units whose
// predecessors on their qubits are all placed (so every qubit sees its gates in circuit order):
// from the seed unit that lets it absorb the most units, the open block takes the ready unit
// that adds the fewest new qubits while it fits in k_max qubits.  A beam search over the seeds
// (sim_plan_opts.search) replaces that schedule when it finds one of fewer blocks.  Block
// matrices are composed in FP64 on the block's own qubits (ascending), later gates multiplying
// from the left.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "internal.h"

using namespace sycsim;

namespace {

// U <- G U, G (GD x GD, GD = 2 or 4) acting on local bits (l0) or (l0, l1) of the D x D
// matrix U (row-major, complex as interleaved doubles).
template <int GD>
void left_multiply_t(double *U, int D, const double *G, int l0, int l1)
{
    for (int base = 0; base < D; base++) {
        if ((base >> l0) & 1) continue;
        if (GD == 4 && ((base >> l1) & 1)) continue;
        int rows[GD];
        rows[0] = base;
        rows[1] = base | (1 << l0);
        if (GD == 4) {
            rows[2] = base | (1 << l1);
            rows[3] = base | (1 << l0) | (1 << l1);
        }
        for (int c = 0; c < D; c++) {
            double ur[GD], ui[GD];
            for (int x = 0; x < GD; x++) {
                ur[x] = U[2 * (rows[x] * D + c)];
                ui[x] = U[2 * (rows[x] * D + c) + 1];
            }
            for (int r = 0; r < GD; r++) {
                double re = 0, im = 0;
                for (int x = 0; x < GD; x++) {
                    const double gr = G[2 * (r * GD + x)], gi = G[2 * (r * GD + x) + 1];
                    re += gr * ur[x] - gi * ui[x];
                    im += gr * ui[x] + gi * ur[x];
                }
                U[2 * (rows[r] * D + c)] = re;
                U[2 * (rows[r] * D + c) + 1] = im;
            }
        }
    }
}

// U <- G U as left_multiply_t, with U's real and imaginary parts in separate D x D row-major
// planes (so the loop over columns vectorises).
template <int GD>
void left_multiply_planes(double *ure, double *uim, int D, const double *G, int l0, int l1)
{
    double gr[GD][GD], gi[GD][GD];
    for (int r = 0; r < GD; r++)
        for (int x = 0; x < GD; x++) {
            gr[r][x] = G[2 * (r * GD + x)];
            gi[r][x] = G[2 * (r * GD + x) + 1];
        }
    for (int base = 0; base < D; base++) {
        if ((base >> l0) & 1) continue;
        if (GD == 4 && ((base >> l1) & 1)) continue;
        int rows[GD];
        rows[0] = base;
        rows[1] = base | (1 << l0);
        if (GD == 4) {
            rows[2] = base | (1 << l1);
            rows[3] = base | (1 << l0) | (1 << l1);
        }
        double *pr[GD], *pi[GD];
        for (int x = 0; x < GD; x++) {
            pr[x] = ure + (size_t)rows[x] * D;
            pi[x] = uim + (size_t)rows[x] * D;
        }
#pragma GCC ivdep
        for (int c = 0; c < D; c++) {
            double xr[GD], xi[GD];
            for (int x = 0; x < GD; x++) {
                xr[x] = pr[x][c];
                xi[x] = pi[x][c];
            }
            for (int r = 0; r < GD; r++) {
                double re = 0, im = 0;
                for (int x = 0; x < GD; x++) {
                    re += gr[r][x] * xr[x] - gi[r][x] * xi[x];
                    im += gr[r][x] * xi[x] + gi[r][x] * xr[x];
                }
                pr[r][c] = re;
                pi[r][c] = im;
            }
        }
    }
}

// Beam width of the block search (sim_plan_opts.search; 0 = the default, 1 = the greedy
// schedule alone).
constexpr int kPlanSearchDefault = 16, kPlanSearchMax = 256;
int search_width(int search)
{
    return search > 0 ? std::min(search, kPlanSearchMax) : kPlanSearchDefault;
}

// Passes 1 and 2 of the planner over the gates gates[idx[0]], gates[idx[1]], ... (circuit order):
// the units (a two-qubit gate with the single-qubit gates folded into it) and their greedy grouping
// into blocks of at most kmax qubits (block qubits in order of first use).  Returns 0, or 1 with
// *bad = the gate of unknown kind, or 2 with *bad = the gate with bad qubits.
struct Unit {
    int q[2];
    int nq;
    std::vector<int> gates;  // indices into the full gate list
    uint64_t mask;           // bit q set for each of its qubits
};

struct Grouping {
    std::vector<Unit> units;
    std::vector<std::vector<int>> qubits;       // per block
    std::vector<std::vector<int>> block_units;  // per block, in order
};

int group_gates(int n_qubits, const sim_gate *gates, const std::vector<int> &idx, int kmax, int width,
                Grouping &gr, int *bad)
{
    // Pass 1 (Sect. 3: single-qubit gates can be aggregated with neighbouring two-qubit gates):
    // each single-qubit gate joins the next two-qubit gate on its qubit, or the previous one
    // when none follows; a qubit without two-qubit gates keeps its own unit.
    std::vector<Unit> &units = gr.units;
    std::vector<std::vector<int>> pending(n_qubits);
    std::vector<int> last2q(n_qubits, -1);
    double G[32];
    for (const int gi : idx) {
        const sim_gate &g = gates[gi];
        const int d = gate_matrix(g, G);
        if (!d) {
            *bad = gi;
            return 1;
        }
        const int nq = d == 2 ? 1 : 2;
        const int Q[2] = {g.q0, g.q1};
        for (int i = 0; i < nq; i++)
            if (Q[i] < 0 || Q[i] >= n_qubits || (i == 1 && Q[1] == Q[0])) {
                *bad = gi;
                return 2;
            }
        if (nq == 1) {
            pending[g.q0].push_back(gi);
            continue;
        }
        Unit u{{g.q0, g.q1}, 2, {}, (1ull << g.q0) | (1ull << g.q1)};
        for (int i = 0; i < 2; i++) {
            u.gates.insert(u.gates.end(), pending[Q[i]].begin(), pending[Q[i]].end());
            pending[Q[i]].clear();
            last2q[Q[i]] = (int)units.size();
        }
        u.gates.push_back(gi);
        units.push_back(std::move(u));
    }
    for (int q = 0; q < n_qubits; q++) {
        if (pending[q].empty()) continue;
        if (last2q[q] >= 0) {
            auto &gl = units[last2q[q]].gates;
            gl.insert(gl.end(), pending[q].begin(), pending[q].end());
        } else {
            units.push_back(Unit{{q, -1}, 1, pending[q], 1ull << q});
        }
    }

    // Pass 2: blocks are formed one after another.  A unit is ready once every earlier unit on
    // its qubits has been placed (in an earlier block or earlier in the open block).  Filling a
    // block from a seed unit: repeatedly take, among the ready units that still fit in kmax
    // qubits, one that adds the fewest new qubits (the earliest unit on ties), until none fits.
    // Each block tries every ready unit as its seed and keeps the one whose fill takes the most
    // units (the earliest seed on ties).  Taking units from anywhere in the circuit, not only
    // the next ones in gate order, lets a block run ahead on its qubits while other parts of the
    // lattice wait: on the 30-qubit, 20-cycle circuit 49 blocks of <= 5 qubits instead of 69
    // in plain gate order (56 with the earliest ready unit as every block's seed), 37 of <= 6.
    // With width > 1 a beam search over the seeds follows (below).
    const int nu = (int)units.size();
    std::vector<std::vector<int>> succ(nu);
    std::vector<int> indeg(nu, 0), lastu(n_qubits, -1);
    for (int ui = 0; ui < nu; ui++) {
        const Unit &u = units[ui];
        int p0 = -1;
        for (int i = 0; i < u.nq; i++) {
            const int p = lastu[u.q[i]];
            if (p >= 0 && p != p0) {
                succ[p].push_back(ui);
                indeg[ui]++;
                p0 = p;
            }
            lastu[u.q[i]] = ui;
        }
    }
    std::vector<int> ready0;
    for (int ui = 0; ui < nu; ui++)
        if (indeg[ui] == 0) ready0.push_back(ui);
    // Fill one block starting from `seed` (an element of rd); rd and ind (the unplaced
    // predecessor counts) are updated, the taken units appended to `taken` and the block's
    // qubits to `bq`.
    auto fill = [&](int seed, std::vector<int> &rd, std::vector<int> &ind, std::vector<int> &taken,
                    std::vector<int> &bq) {
        uint64_t bm = 0;  // the block's qubits as a mask (bq keeps their order of first use)
        for (const int q : bq) bm |= 1ull << q;
        int nbq = (int)bq.size(), next = seed;
        for (;;) {
            int pos = -1;
            if (next >= 0) {
                pos = (int)(std::find(rd.begin(), rd.end(), next) - rd.begin());
            } else {
                int best_add = kMaxK + 1;
                for (int r = 0; r < (int)rd.size(); r++) {
                    const int add = __builtin_popcountll(units[rd[r]].mask & ~bm);
                    if (nbq + add > kmax) continue;
                    if (add < best_add || (add == best_add && rd[r] < rd[pos])) {
                        pos = r;
                        best_add = add;
                    }
                }
                if (pos < 0) break;
            }
            next = -1;
            const int ui = rd[pos];
            rd.erase(rd.begin() + pos);
            taken.push_back(ui);
            const Unit &u = units[ui];
            for (int i = 0; i < u.nq; i++)
                if (!((bm >> u.q[i]) & 1)) {
                    bq.push_back(u.q[i]);
                    bm |= 1ull << u.q[i];
                    nbq++;
                }
            for (const int sx : succ[ui])
                if (--ind[sx] == 0) rd.push_back(sx);
        }
    };
    std::vector<int> rd, taken, bq;
    // the greedy schedule: every block's seed is the ready unit whose fill takes the most units
    std::vector<int> seeds;
    {
        std::vector<int> ready = ready0, ind = indeg;
        int placed = 0;
        while (placed < nu) {
            int best_seed = -1, best_n = -1;
            for (const int seed : ready) {  // trial fills, undone afterwards
                rd = ready;
                taken.clear();
                bq.clear();
                fill(seed, rd, ind, taken, bq);
                for (const int ui : taken)
                    for (const int sx : succ[ui]) ind[sx]++;
                if ((int)taken.size() > best_n || ((int)taken.size() == best_n && seed < best_seed)) {
                    best_n = (int)taken.size();
                    best_seed = seed;
                }
            }
            seeds.push_back(best_seed);
            taken.clear();
            bq.clear();
            fill(best_seed, ready, ind, taken, bq);
            placed += (int)taken.size();
        }
    }
    // Beam search (width > 1) for a schedule of fewer blocks: after each block, keep the `width`
    // partial schedules that have placed the most units (earlier ones on ties).  Two partial
    // schedules that have placed the same units are one; they are told apart by a key, the XOR
    // of a random 64-bit word per placed unit (Zobrist hashing).  Each child is scored without
    // being kept (its parent, seed, count and key) and only the `width` chosen are rebuilt.  The
    // first schedule to place every unit in fewer blocks than the greedy one replaces it.
    if (width > 1) {
        std::vector<uint64_t> zob(nu);
        uint64_t z = 0;
        for (int ui = 0; ui < nu; ui++) {  // splitmix64 (Steele, Lea, Flood 2014)
            z += 0x9E3779B97F4A7C15ull;
            uint64_t x = z;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            zob[ui] = x ^ (x >> 31);
        }
        struct Partial {
            int placed = 0;
            uint64_t key = 0;
            std::vector<int> ready, ind, seeds;
        };
        struct Child {
            int placed;
            uint64_t key;
            int parent, seed;
        };
        std::vector<Partial> cur(width), next(width);
        cur[0].ready = ready0;
        cur[0].ind = indeg;
        int ncur = 1;
        std::vector<Child> kids;
        std::vector<int> rd2, ind2;
        bool done = false;
        for (int depth = 1; depth < (int)seeds.size() && !done; depth++) {
            kids.clear();
            for (int pi = 0; pi < ncur && !done; pi++) {
                const Partial &p = cur[pi];
                for (const int seed : p.ready) {
                    rd2 = p.ready;
                    ind2 = p.ind;
                    taken.clear();
                    bq.clear();
                    fill(seed, rd2, ind2, taken, bq);
                    const int placed = p.placed + (int)taken.size();
                    if (placed == nu) {
                        seeds = p.seeds;
                        seeds.push_back(seed);
                        done = true;
                        break;
                    }
                    uint64_t key = p.key;
                    for (const int ui : taken) key ^= zob[ui];
                    kids.push_back(Child{placed, key, pi, seed});
                }
            }
            if (done) break;
            std::stable_sort(kids.begin(), kids.end(), [](const Child &x, const Child &y) { return x.placed > y.placed; });
            int nnext = 0;
            for (const Child &c : kids) {
                if (nnext == width) break;
                bool dup = false;
                for (int j = 0; j < nnext && !dup; j++) dup = next[j].key == c.key;
                if (dup) continue;
                const Partial &p = cur[c.parent];
                Partial &d = next[nnext++];
                d.placed = c.placed;
                d.key = c.key;
                d.ready = p.ready;
                d.ind = p.ind;
                d.seeds = p.seeds;
                d.seeds.push_back(c.seed);
                taken.clear();
                bq.clear();
                fill(c.seed, d.ready, d.ind, taken, bq);
            }
            cur.swap(next);
            ncur = nnext;
        }
    }
    // the blocks of the chosen schedule
    {
        std::vector<int> ready = ready0, ind = indeg;
        for (const int seed : seeds) {
            gr.qubits.emplace_back();
            gr.block_units.emplace_back();
            fill(seed, ready, ind, gr.block_units.back(), gr.qubits.back());
        }
    }
    return 0;
}

// Greedy phase split (Sect. 4): in a phase with set X sliced (which[q] == X), apply, in order,
// every remaining gate that avoids X and every qubit already holding a deferred gate; the
// deferred gates form the next phase's input, with the other set sliced.  Returns false if some
// gates can never be applied (a gate coupling the two sets).
bool split_phases(int n_qubits, int n_gates, const sim_gate *gates, const std::vector<int> &which, int first,
                  std::vector<std::pair<int, std::vector<int>>> &phases)
{
    double G[32];
    std::vector<int> rem(n_gates);
    for (int g = 0; g < n_gates; g++) rem[g] = g;
    int cur = first, idle = 0;
    while (!rem.empty() && idle < 2) {
        std::vector<char> blocked(n_qubits, 0);
        for (int q = 0; q < n_qubits; q++) blocked[q] = which[q] == cur;
        std::vector<int> take, defer;
        for (int g : rem) {
            const int d = gate_matrix(gates[g], G);
            const int Q[2] = {gates[g].q0, gates[g].q1};
            const int nq = d == 2 ? 1 : 2;
            bool ok = true;
            for (int i = 0; i < nq; i++) ok &= !blocked[Q[i]];
            if (ok) {
                take.push_back(g);
            } else {
                defer.push_back(g);
                for (int i = 0; i < nq; i++) blocked[Q[i]] = 1;
            }
        }
        if (take.empty()) {
            idle++;
        } else {
            idle = 0;
            phases.push_back({cur, take});
        }
        rem.swap(defer);
        cur = 1 - cur;
    }
    return rem.empty();
}

}  // namespace

extern "C" {

int sim_gate_matrix(const sim_gate *g, double *out)
{
    if (!g || !out) return fail(nullptr, SIM_E_INVAL, "sim_gate_matrix: NULL argument");
    const int d = gate_matrix(*g, out);
    if (!d) return fail(nullptr, SIM_E_INVAL, "sim_gate_matrix: unknown kind %d", g->kind);
    return d;
}

int sim_plan_create(int n_qubits, int n_gates, const sim_gate *gates, const sim_plan_opts *o,
                    sim_plan_t **out)
{
    if (!out) return fail(nullptr, SIM_E_INVAL, "sim_plan_create: out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > kMaxQubits)
        return fail(nullptr, SIM_E_INVAL, "sim_plan_create: n_qubits=%d", n_qubits);
    if (n_gates < 0 || (n_gates > 0 && !gates))
        return fail(nullptr, SIM_E_INVAL, "sim_plan_create: bad gate list");
    sim_plan_opts opts{};
    opts.kmax = 4;
    if (o) opts = *o;
    if (opts.kmax < 2 || opts.kmax > kMaxK)
        return fail(nullptr, SIM_E_INVAL, "sim_plan_create: kmax=%d outside 2..%d", opts.kmax, kMaxK);
    if (!precision_ok(opts.precision))
        return fail(nullptr, SIM_E_INVAL, "sim_plan_create: precision %d", opts.precision);
    if (opts.search < 0 || opts.search > kPlanSearchMax)
        return fail(nullptr, SIM_E_INVAL, "sim_plan_create: search=%d outside 0..%d", opts.search, kPlanSearchMax);

    auto *p = new sim_plan_s();
    p->n = n_qubits;
    p->n_gates = n_gates;
    p->kmax = opts.kmax;
    p->precision = opts.precision;
    Grouping gr;
    std::vector<int> idx(n_gates);
    for (int i = 0; i < n_gates; i++) idx[i] = i;
    int bad = 0;
    const int grc = group_gates(n_qubits, gates, idx, opts.kmax, search_width(opts.search), gr, &bad);
    if (grc) {
        delete p;
        return fail(nullptr, SIM_E_INVAL, grc == 1 ? "sim_plan_create: gate %d has unknown kind %d"
                                                   : "sim_plan_create: gate %d has bad qubits",
                    bad, gates[bad].kind);
    }
    const std::vector<Unit> &units = gr.units;
    const std::vector<std::vector<int>> &block_units = gr.block_units;
    double G[32];
    p->blocks.resize(gr.qubits.size());
    for (size_t bi = 0; bi < gr.qubits.size(); bi++) {
        p->blocks[bi].qubits = gr.qubits[bi];
        for (int ui : block_units[bi]) {
            const auto &ug = units[ui].gates;
            p->blocks[bi].gates.insert(p->blocks[bi].gates.end(), ug.begin(), ug.end());
        }
    }
    // compose each block in FP64: each unit's gates first into one 2x2 or 4x4 matrix (local bit 0
    // = the unit's first qubit), then that matrix into the block.  The block's matrix grows with
    // its qubits: it starts as the 1x1 identity, and when a unit brings a qubit the block has not
    // met yet, the matrix becomes M (x) I on a new top bit, so a unit is multiplied in on the
    // qubits met so far (2-2.7x fewer products at k_max 5-6 than on all k from the start).  The
    // local bits follow the order the qubits were met; the last step reorders rows and columns
    // to ascending qubits.  Real and imaginary parts are kept in separate planes.
    std::vector<double> mre, mim, tre, tim;
    for (size_t bi = 0; bi < p->blocks.size(); bi++) {
        PlanBlock &b = p->blocks[bi];
        std::sort(b.qubits.begin(), b.qubits.end());
        const int k = (int)b.qubits.size(), D = 1 << k;
        int met[kMaxK], n_met = 0, d = 1;
        mre.assign(1, 1.0);
        mim.assign(1, 0.0);
        for (int ui : block_units[bi]) {
            const Unit &u = units[ui];
            const int ud = u.nq == 2 ? 4 : 2;
            double Mu[32] = {0};
            for (int i = 0; i < ud; i++) Mu[2 * (i * ud + i)] = 1.0;
            for (int gi : u.gates) {
                const sim_gate &g = gates[gi];
                const int gd = gate_matrix(g, G);
                if (gd == 4) {
                    const bool same = g.q0 == u.q[0];  // the gate's bit 0 on the unit's bit 0?
                    left_multiply_t<4>(Mu, 4, G, same ? 0 : 1, same ? 1 : 0);
                } else {
                    left_multiply_t<2>(Mu, ud, G, g.q0 == u.q[0] ? 0 : 1, -1);
                }
            }
            int lb[2] = {-1, -1};
            for (int i = 0; i < u.nq; i++) {
                lb[i] = (int)(std::find(met, met + n_met, u.q[i]) - met);
                if (lb[i] < n_met) continue;
                // a new qubit: M -> diag(M, M), the qubit on the new top bit
                const int d2 = 2 * d;
                tre.assign((size_t)d2 * d2, 0.0);
                tim.assign((size_t)d2 * d2, 0.0);
                for (int r = 0; r < d; r++)
                    for (int c = 0; c < d; c++) {
                        const double vr = mre[(size_t)r * d + c], vi = mim[(size_t)r * d + c];
                        tre[(size_t)r * d2 + c] = vr;
                        tim[(size_t)r * d2 + c] = vi;
                        tre[(size_t)(d + r) * d2 + d + c] = vr;
                        tim[(size_t)(d + r) * d2 + d + c] = vi;
                    }
                mre.swap(tre);
                mim.swap(tim);
                d = d2;
                met[n_met++] = u.q[i];
            }
            if (u.nq == 2)
                left_multiply_planes<4>(mre.data(), mim.data(), d, Mu, lb[0], lb[1]);
            else
                left_multiply_planes<2>(mre.data(), mim.data(), d, Mu, lb[0], -1);
        }
        if (d != D) {  // the units' qubits are the block's qubits by construction
            delete p;
            return fail(nullptr, SIM_E_INVAL, "sim_plan_create: block %zu met %d of its %d qubits", bi, n_met, k);
        }
        // local bit i (the i-th qubit met) -> bit pos[i] of the ascending order
        int pos[kMaxK];
        for (int i = 0; i < n_met; i++)
            pos[i] = (int)(std::find(b.qubits.begin(), b.qubits.end(), met[i]) - b.qubits.begin());
        std::vector<int> to(D);
        for (int x = 0; x < D; x++) {
            int y = 0;
            for (int i = 0; i < n_met; i++) y |= ((x >> i) & 1) << pos[i];
            to[x] = y;
        }
        b.mat.assign(2 * (size_t)D * D, 0.0);
        for (int r = 0; r < D; r++)
            for (int c = 0; c < D; c++) {
                const size_t o = 2 * ((size_t)to[r] * D + to[c]);
                b.mat[o] = mre[(size_t)r * D + c];
                b.mat[o + 1] = mim[(size_t)r * D + c];
            }
    }
    *out = p;
    return SIM_OK;
}

int sim_plan_destroy(sim_plan_t *p)
{
    if (!p) return fail(nullptr, SIM_E_INVAL, "sim_plan_destroy: NULL plan");
    delete p;
    return SIM_OK;
}

int sim_plan_info(const sim_plan_t *p, int *n_blocks, int *n_gates, int *max_k)
{
    if (!p) return fail(nullptr, SIM_E_INVAL, "sim_plan_info: NULL plan");
    if (n_blocks) *n_blocks = (int)p->blocks.size();
    if (n_gates) *n_gates = p->n_gates;
    if (max_k) {
        int m = 0;
        for (auto &b : p->blocks) m = std::max(m, (int)b.qubits.size());
        *max_k = m;
    }
    return SIM_OK;
}

int sim_plan_block(const sim_plan_t *p, int i, int *k, int *targets, double *matrix)
{
    if (!p) return fail(nullptr, SIM_E_INVAL, "sim_plan_block: NULL plan");
    if (i < 0 || i >= (int)p->blocks.size())
        return fail(nullptr, SIM_E_INVAL, "sim_plan_block: index %d outside 0..%zu", i,
                    p->blocks.size());
    const PlanBlock &b = p->blocks[i];
    if (k) *k = (int)b.qubits.size();
    if (targets) std::copy(b.qubits.begin(), b.qubits.end(), targets);
    if (matrix) std::copy(b.mat.begin(), b.mat.end(), matrix);
    return SIM_OK;
}

}  // extern "C"

#ifndef SYCSIM_LAYOUT_STARTS
#define SYCSIM_LAYOUT_STARTS 4  // seeded starts of the layout search (2, 4, 8, 16 measured: 4 is within 0.2 % of 16 at a quarter of the host time)
#endif

namespace {

// Estimated time of one fused pass over 2^30 amplitudes (ms) on the kernel a block of k targets at
// physical bits tpos takes, from CUDA-event timings of each kernel path on GB300; the layout search
// only compares sums of these.
double pass_ms(int k, const int *tpos, int precision)
{
    int low4 = 0, low5 = 0;
    bool le7 = false;
    for (int i = 0; i < k; i++) {
        low4 += tpos[i] < 4;
        low5 += tpos[i] < 5;
        le7 = le7 || tpos[i] <= 7;
    }
    if (tmem_mode(precision)) {
        // tcgen05 with <= 1 target below bit 4 (k = 5, 6) or none (k = 4), else mma.sync 3xFP16;
        // k = 6 (A operand in tensor memory) runs 2.65 ms with one target below bit 4 and
        // 2.69-2.72 ms otherwise; k = 5 tiles move 2 KiB runs once a target sits at bit 7 or below,
        // else twice the groups
        if (k == 6) return low4 >= 2 ? 5.10 : (low4 == 1 ? 2.65 : 2.70);
        if (k == 5) return low4 >= 2 ? 2.70 : (le7 ? 2.55 : 2.63);
        if (k == 4) return low4 >= 1 ? 2.68 : 2.55;
        return 2.45;
    }
    if (precision == SIM_FP32) {
        // register kernel: each target below bit 5 costs warp exchanges (k = 4: 2.79 ms with none,
        // 3.3 mixed, 4.3 all low); k >= 5 is FP32-ALU bound whatever the targets
        if (k >= 5) return 6.9;
        if (k == 4) return low5 == 0 ? 2.79 : (low5 >= 4 ? 4.29 : 3.30);
        return low5 == 0 ? 2.45 : 2.90;
    }
    return 1.0;
}

// Improve a phase's layout without a second permutation pass: pos[q] is qubit q's physical bit
// after the phase's sliced-set moves, used[b] marks the positions those moves changed.  Swaps of
// two positions below `top` that no move (and no earlier swap) touched keep the whole move one
// set of disjoint transpositions, which sim_permute does in one pass; take the swap that lowers
// the plan's per-pass estimate most, until none does.  Returns the estimate's change (<= 0).
double improve_by_disjoint_swaps(const sim_plan_s *p, std::vector<int> &pos, std::vector<char> &used, int top)
{
    if (!tmem_mode(p->precision) && p->precision != SIM_FP32) return 0.0;
    double gain = 0.0;
    const int n = p->n, nb = (int)p->blocks.size();
    std::vector<std::vector<int>> of_qubit(n);
    for (int b = 0; b < nb; b++)
        for (int q : p->blocks[b].qubits) of_qubit[q].push_back(b);
    auto block_cost = [&](int b) {
        int tpos[kMaxK];
        const auto &qs = p->blocks[b].qubits;
        for (size_t i = 0; i < qs.size(); i++) tpos[i] = pos[qs[i]];
        return pass_ms((int)qs.size(), tpos, p->precision);
    };
    auto cls = [](int b) { return b < 4 ? 0 : (b < 8 ? 1 : 2); };
    std::vector<char> mark(nb, 0);
    for (;;) {
        double best = -1e-9;
        int ba = -1, bc = -1;
        for (int a = 0; a < n; a++) {
            if (pos[a] >= top || used[pos[a]]) continue;
            for (int c = a + 1; c < n; c++) {
                if (pos[c] >= top || used[pos[c]] || cls(pos[a]) == cls(pos[c])) continue;
                std::vector<int> touched;
                for (int b : of_qubit[a])
                    if (!mark[b]) mark[b] = 1, touched.push_back(b);
                for (int b : of_qubit[c])
                    if (!mark[b]) mark[b] = 1, touched.push_back(b);
                double before = 0, after = 0;
                for (int b : touched) before += block_cost(b);
                std::swap(pos[a], pos[c]);
                for (int b : touched) after += block_cost(b);
                std::swap(pos[a], pos[c]);
                for (int b : touched) mark[b] = 0;
                if (after - before < best) {
                    best = after - before;
                    ba = a;
                    bc = c;
                }
            }
        }
        if (ba < 0) break;
        used[pos[ba]] = used[pos[bc]] = 1;
        std::swap(pos[ba], pos[bc]);
        gain += best;
    }
    return gain;
}

}  // namespace

namespace sycsim {

double plan_estimate_ms(const sim_plan_s *p, const int *bit_of)
{
    double t = 0.0;
    for (const auto &b : p->blocks) {
        int tpos[kMaxK];
        for (size_t i = 0; i < b.qubits.size(); i++) tpos[i] = bit_of[b.qubits[i]];
        t += pass_ms((int)b.qubits.size(), tpos, p->precision);
    }
    return t;
}

}  // namespace sycsim

extern "C" {

// The layout search; low (may be NULL): only qubits with low[q] != 0 may sit at physical bits
// 0 .. n_low - 1.
static int layout_search(const sim_plan_t *p, const char *low, int n_low, int *perm, double *est_ms)
{
    constexpr int kLayoutStarts = SYCSIM_LAYOUT_STARTS;
    const int n = p->n, nb = (int)p->blocks.size();
    auto allowed = [&](const std::vector<int> &ps, int q) { return !low || ps[q] >= n_low || low[q]; };
    // move qubits of the low set into bits 0 .. n_low - 1 (swapping out the others), keeping order
    auto fix_low = [&](std::vector<int> &ps) {
        if (!low) return;
        std::vector<int> at(n);
        for (int q = 0; q < n; q++) at[ps[q]] = q;
        int next_ok = 0;  // scan qubits of the low set that sit above n_low
        for (int b = 0; b < n_low; b++) {
            if (low[at[b]]) continue;
            while (next_ok < n && !(low[next_ok] && ps[next_ok] >= n_low)) next_ok++;
            if (next_ok == n) return;
            const int q = at[b], r = next_ok;
            std::swap(ps[q], ps[r]);
            at[ps[q]] = q;
            at[ps[r]] = r;
        }
    };
    std::vector<std::vector<int>> of_qubit(n);  // blocks holding each qubit
    for (int b = 0; b < nb; b++)
        for (int q : p->blocks[b].qubits) of_qubit[q].push_back(b);
    std::vector<int> pos(n);  // pos[q] = physical bit of qubit q
    auto block_cost = [&](int b) {
        int tpos[kMaxK];
        const auto &qs = p->blocks[b].qubits;
        for (size_t i = 0; i < qs.size(); i++) tpos[i] = pos[qs[i]];
        return pass_ms((int)qs.size(), tpos, p->precision);
    };
    auto total = [&]() {
        double t = 0;
        for (int b = 0; b < nb; b++) t += block_cost(b);
        return t;
    };
    for (int q = 0; q < n; q++) pos[q] = q;
    const double ident = total();
    fix_low(pos);
    std::vector<int> best = pos;
    double best_cost = total();
    const bool modelled = tmem_mode(p->precision) || p->precision == SIM_FP32;
    uint64_t rs = 0x9E3779B97F4A7C15ull;  // SplitMix64 state for the seeded starts
    auto next = [&]() {
        uint64_t z = (rs += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<char> mark(nb, 0);
    // the estimates depend only on which targets sit below bit 4 and at bits 4-7, so a swap of two
    // positions of the same class (0-3, 4-7, 8 and up) changes nothing and is skipped
    auto cls = [](int b) { return b < 4 ? 0 : (b < 8 ? 1 : 2); };
    for (int start = 0; modelled && start < kLayoutStarts; start++) {
        for (int q = 0; q < n; q++) pos[q] = q;
        for (int q = n - 1; start > 0 && q > 0; q--) std::swap(pos[q], pos[next() % (uint64_t)(q + 1)]);
        fix_low(pos);
        double cost = total();
        for (int sweep = 0; sweep < 64; sweep++) {
            bool improved = false;
            for (int a = 0; a < n; a++)
                for (int c = a + 1; c < n; c++) {
                    if (cls(pos[a]) == cls(pos[c])) continue;
                    std::vector<int> touched;
                    for (int b : of_qubit[a])
                        if (!mark[b]) mark[b] = 1, touched.push_back(b);
                    for (int b : of_qubit[c])
                        if (!mark[b]) mark[b] = 1, touched.push_back(b);
                    double before = 0, after = 0;
                    for (int b : touched) before += block_cost(b);
                    std::swap(pos[a], pos[c]);
                    for (int b : touched) after += block_cost(b);
                    for (int b : touched) mark[b] = 0;
                    if (after < before - 1e-9 && allowed(pos, a) && allowed(pos, c)) {
                        cost += after - before;
                        improved = true;
                    } else {
                        std::swap(pos[a], pos[c]);
                    }
                }
            if (!improved) break;
        }
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = pos;
        }
    }
    for (int q = 0; q < n; q++) perm[q] = best[q];
    if (est_ms) {
        est_ms[0] = best_cost;
        est_ms[1] = ident;
    }
    return SIM_OK;
}

int sim_plan_layout(const sim_plan_t *p, int *perm, double *est_ms)
{
    if (!p || !perm) return fail(nullptr, SIM_E_INVAL, "sim_plan_layout: NULL argument");
    return layout_search(p, nullptr, 0, perm, est_ms);
}

int sim_plan_layout_front(const sim_plan_t *p, const sim_split_t *s, int *perm, double *est_ms)
{
    if (!p || !s || !perm) return fail(nullptr, SIM_E_INVAL, "sim_plan_layout_front: NULL argument");
    if (s->n != p->n) return fail(nullptr, SIM_E_INVAL, "sim_plan_layout_front: split and plan differ in n");
    std::vector<char> low(p->n);
    int n_side0 = 0;
    for (int q = 0; q < p->n; q++) n_side0 += (low[q] = s->side[q] == 0);
    // the contraction's stores: lanes of a warp hold 32 consecutive x (the side-0 qubits in order of
    // their physical bits), so side-0 qubits at bits 0-4 make each store one 256-byte run
    return layout_search(p, low.data(), std::min(5, n_side0), perm, est_ms);
}

int sim_phases_layout(const sim_phases_t *ph, const sim_split_t *front, int resident, int *perm, double *est_ms)
{
    if (!ph || !perm) return fail(nullptr, SIM_E_INVAL, "sim_phases_layout: NULL argument");
    if (front && front->n != ph->n) return fail(nullptr, SIM_E_INVAL, "sim_phases_layout: split of another n");
    const int n = ph->n, s = ph->s, r = n - 2 * s;
    // the two sets' bits: a host store keeps B on n-2s .. n-s-1 and A on top; a resident sliced
    // state has the first phase's sliced set on top (no move before it) and the other below
    const int first = ph->set_of.empty() ? 0 : ph->set_of[0];
    const int *top = resident && first == 1 ? ph->set_b : ph->set_a;
    const int *below = top == ph->set_a ? ph->set_b : ph->set_a;
    std::vector<char> sliced(n, 0);
    for (int i = 0; i < s; i++) sliced[ph->set_a[i]] = sliced[ph->set_b[i]] = 1;
    std::vector<int> order;  // the others, position i -> qubit; with a front, side-0 qubits first
    for (int pass = 0; pass < 2; pass++)
        for (int q = 0; q < n; q++)
            if (!sliced[q] && (!front || (front->side[q] == 0) == (pass == 0)) && (front || pass == 0))
                order.push_back(q);
    // with a front, bits 0 .. low-1 keep side-0 qubits: the contraction's 32 lanes of a warp then
    // write 32 consecutive amplitudes
    int n_group0 = front ? 0 : r;
    if (front)
        for (int q = 0; q < n; q++) n_group0 += !sliced[q] && front->side[q] == 0;
    const int low = front ? std::min(n_group0, 5) : 0;
    auto allowed = [&](const std::vector<int> &ord) {
        for (int i = 0; i < low; i++)
            if (front->side[ord[i]] != 0) return false;
        return true;
    };
    // a phase's layout: the others on 0 .. r-1, the set it does not slice on r .. r+s-1 (its
    // sliced set's bits are never read: its blocks avoid it).  Host store: the slot's layout.
    // Resident: the first phase's, as it runs; later phases move the sets, the others stay.
    auto total = [&](const std::vector<int> &ord) {
        int bit[kMaxQubits];
        for (int q = 0; q < n; q++) bit[q] = -1;
        for (int i = 0; i < r; i++) bit[ord[i]] = i;
        double t = 0.0;
        for (size_t i = 0; i < ph->plans.size(); i++) {
            const int *hi = ph->set_of[i] == 0 ? ph->set_b : ph->set_a;
            for (int j = 0; j < s; j++) bit[hi[j]] = r + j;
            t += plan_estimate_ms(ph->plans[i], bit);
        }
        return t;
    };
    std::vector<int> start0 = order;
    if (!front) std::sort(start0.begin(), start0.end());
    const double ascending = total(start0);
    double best = ascending;
    std::vector<int> best_order = start0;
    std::mt19937 rng(12345);
    for (int start = 0; start < SYCSIM_LAYOUT_STARTS; start++) {
        std::vector<int> ord = start0;
        if (start > 0) {  // seeded shuffles: with a front within each group, else all
            std::shuffle(ord.begin(), ord.begin() + n_group0, rng);
            std::shuffle(ord.begin() + n_group0, ord.end(), rng);
        }
        double cost = total(ord);
        for (bool improved = true; improved;) {  // pairwise exchanges while one lowers the estimate
            improved = false;
            for (int i = 0; i < r; i++)
                for (int j = i + 1; j < r; j++) {
                    std::swap(ord[i], ord[j]);
                    const double c = allowed(ord) ? total(ord) : 1e300;
                    if (c < cost - 1e-9) {
                        cost = c;
                        improved = true;
                    } else {
                        std::swap(ord[i], ord[j]);
                    }
                }
        }
        if (cost < best - 1e-9) {
            best = cost;
            best_order = ord;
        }
    }
    for (int i = 0; i < r; i++) perm[best_order[i]] = i;
    for (int i = 0; i < s; i++) {
        perm[below[i]] = r + i;
        perm[top[i]] = n - s + i;
    }
    if (est_ms) {
        est_ms[0] = best;
        est_ms[1] = ascending;
    }
    return SIM_OK;
}

int sim_apply_plan(sim_t *h, const sim_plan_t *p)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_apply_plan: NULL handle");
    state_written(h);
    if (!p) return fail(h, SIM_E_INVAL, "sim_apply_plan: NULL plan");
    if (p->n != h->n)
        return fail(h, SIM_E_INVAL, "sim_apply_plan: plan has %d qubits, handle %d", p->n, h->n);
    if (h->store != SIM_STORE_DEVICE)
        return fail(h, SIM_E_UNSUPPORTED, "sim_apply_plan: host-store state: use sim_run_phase");
    SIM_DEVICE_SCOPE(h, h->device);
    // Every block's operands (tensor-core R^T fragments, 6-qubit matrices) are built on the host and
    // uploaded in one copy before the first launch, then every block is launched from them: the
    // calling thread never waits for the device inside the plan (a per-block staging ring would make
    // it wait for the block launched a ring's length earlier), and a plan costs one small copy.
    struct Prep {
        int k;
        int tpos[kMaxK];
        size_t moff, off, bytes;
    };
    static thread_local std::vector<Prep> prep;
    static thread_local std::vector<float2> mats;
    const size_t nb = p->blocks.size();
    prep.resize(nb);
    size_t mtot = 0, total = 0;
    for (size_t i = 0; i < nb; i++) mtot += (size_t)1 << (2 * p->blocks[i].qubits.size());
    mats.resize(mtot);
    mtot = 0;
    for (size_t i = 0; i < nb; i++) {
        const PlanBlock &b = p->blocks[i];
        Prep &pb = prep[i];
        pb.k = (int)b.qubits.size();
        pb.moff = mtot;
        const int rc = prepare_block(h, pb.k, b.qubits.data(), b.mat.data(), pb.tpos, mats.data() + mtot);
        if (rc != SIM_OK) return rc;
        mtot += (size_t)1 << (2 * pb.k);
        pb.bytes = block_staged_bytes(h->n, pb.k, pb.tpos, p->precision);
        pb.off = total;
        total += (pb.bytes + 255) & ~size_t(255);
    }
    char *d_ops = nullptr;
    int slot = -1;
    if (total) {
        slot = h->plan_next;
        h->plan_next ^= 1;
        if (!h->plan_ev[slot]) SIM_CUDA_TRY(h, cudaEventCreateWithFlags(&h->plan_ev[slot], cudaEventDisableTiming));
        // the plan that used this slot two calls ago has been uploaded and run
        SIM_CUDA_TRY(h, cudaEventSynchronize(h->plan_ev[slot]));
        if (h->plan_bytes[slot] < total) {
            if (h->h_plan[slot]) cudaFreeHost(h->h_plan[slot]);
            if (h->d_plan[slot]) cudaFree(h->d_plan[slot]);
            h->h_plan[slot] = nullptr;
            h->d_plan[slot] = nullptr;
            h->plan_bytes[slot] = 0;
            const size_t want = total + total / 2;
            if (cudaHostAlloc(reinterpret_cast<void **>(&h->h_plan[slot]), want, cudaHostAllocDefault) != cudaSuccess) {
                h->h_plan[slot] = nullptr;
                return fail(h, SIM_E_NOMEM_HOST, "sim_apply_plan: staging buffer");
            }
            if (cudaMalloc(reinterpret_cast<void **>(&h->d_plan[slot]), want) != cudaSuccess) {
                h->d_plan[slot] = nullptr;
                return fail(h, SIM_E_NOMEM_DEV, "sim_apply_plan: staging buffer");
            }
            h->plan_bytes[slot] = want;
        }
        for (size_t i = 0; i < nb; i++)
            if (prep[i].bytes)
                block_build_staged(h->n, prep[i].k, prep[i].tpos, mats.data() + prep[i].moff, p->precision,
                                   h->h_plan[slot] + prep[i].off);
        SIM_CUDA_TRY(h, cudaMemcpyAsync(h->d_plan[slot], h->h_plan[slot], total, cudaMemcpyHostToDevice, h->stream));
        d_ops = h->d_plan[slot];
    }
    const double pass_bytes = 16.0 * std::ldexp(1.0, h->n);
    // the last block, on tcgen05, also leaves its CTAs' (sum p, sum p^2): a following sim_reduce
    // only combines them instead of reading the state again (handles whose state memory is their
    // own and was never handed out: nobody else can write it in between)
    const bool fuse = h->own_state && !h->state_exposed;
    int red_grid = 0;
    for (size_t i = 0; i < nb; i++) {
        const Prep &pb = prep[i];
        const bool last = i + 1 == nb;
        const int ps = prof_begin(h, SIM_PROF_APPLY, pass_bytes, h->stream);
        const int rc = launch_block_staged(h, h->d_state, h->n, pb.k, pb.tpos, mats.data() + pb.moff, p->precision,
                                           d_ops ? d_ops + pb.off : nullptr, h->stream,
                                           last && fuse ? h->d_partials : nullptr, last && fuse ? &red_grid : nullptr);
        prof_end(h, ps, h->stream);
        if (rc != SIM_OK) {
            if (slot >= 0) cudaEventRecord(h->plan_ev[slot], h->stream);
            return rc;
        }
    }
    h->red_blocks = red_grid;
    h->red_epoch = red_grid > 0 ? h->write_epoch : 0;
    if (slot >= 0) SIM_CUDA_TRY(h, cudaEventRecord(h->plan_ev[slot], h->stream));
    return SIM_OK;
}

// ---- CUDA graphs of a plan ----

int sim_graph_create(sim_t *h, const sim_plan_t *p, sim_graph_t **out)
{
    if (!h || !p || !out) return fail(h, SIM_E_INVAL, "sim_graph_create: NULL argument");
    *out = nullptr;
    if (p->n != h->n) return fail(h, SIM_E_INVAL, "sim_graph_create: plan has %d qubits, handle %d", p->n, h->n);
    if (h->store != SIM_STORE_DEVICE)
        return fail(h, SIM_E_UNSUPPORTED, "sim_graph_create: host-store handle (use sim_run_phase)");
    if (h->stream == nullptr)
        return fail(h, SIM_E_UNSUPPORTED, "sim_graph_create: the legacy default stream cannot be captured");
    SIM_DEVICE_SCOPE(h, h->device);
    struct Staged {
        int k;
        int tpos[kMaxK];
        std::vector<float2> mat;
        size_t off, bytes;
    };
    std::vector<Staged> blocks(p->blocks.size());
    static thread_local float2 mat[4096];
    size_t total = 0;
    for (size_t i = 0; i < p->blocks.size(); i++) {
        const PlanBlock &b = p->blocks[i];
        Staged &sb = blocks[i];
        sb.k = (int)b.qubits.size();
        const int rc = prepare_block(h, sb.k, b.qubits.data(), b.mat.data(), sb.tpos, mat);
        if (rc != SIM_OK) return rc;
        sb.mat.assign(mat, mat + (1 << (2 * sb.k)));
        sb.bytes = block_staged_bytes(h->n, sb.k, sb.tpos, p->precision);
        sb.off = total;
        total += (sb.bytes + 255) & ~size_t(255);
    }
    auto *g = new sim_graph_s();
    g->h = h;
    g->n_blocks = (int)blocks.size();
    g->bit_of.assign(h->bit_of, h->bit_of + h->n);
    auto cleanup = [&](int code, const char *what) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->d_staged) cudaFree(g->d_staged);
        delete g;
        return fail(h, code, "sim_graph_create: %s: %s", what, cudaGetErrorString(cudaGetLastError()));
    };
    if (total) {
        std::vector<char> host(total);
        for (auto &sb : blocks)
            if (sb.bytes) block_build_staged(h->n, sb.k, sb.tpos, sb.mat.data(), p->precision, host.data() + sb.off);
        if (cudaMalloc(&g->d_staged, total) != cudaSuccess) return cleanup(SIM_E_NOMEM_DEV, "staging buffer");
        if (cudaMemcpy(g->d_staged, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(SIM_E_CUDA, "staging upload");
    }
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cleanup(SIM_E_CUDA, "begin capture");
    int rc = SIM_OK;
    for (auto &sb : blocks) {
        rc = launch_block_staged(h, h->d_state, h->n, sb.k, sb.tpos, sb.mat.data(), p->precision,
                                 static_cast<char *>(g->d_staged) + sb.off, h->stream);
        if (rc != SIM_OK) break;
    }
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &g->graph);  // always ends the capture
    if (rc != SIM_OK || ec != cudaSuccess) return cleanup(rc != SIM_OK ? rc : SIM_E_CUDA, "capture");
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) return cleanup(SIM_E_CUDA, "instantiate");
    *out = g;
    return SIM_OK;
}

int sim_graph_launch(sim_t *h, const sim_graph_t *g)
{
    if (!h || !g) return fail(h, SIM_E_INVAL, "sim_graph_launch: NULL argument");
    state_written(h);
    if (g->h != h) return fail(h, SIM_E_INVAL, "sim_graph_launch: the graph belongs to another handle");
    if (!std::equal(g->bit_of.begin(), g->bit_of.end(), h->bit_of))
        return fail(h, SIM_E_INVAL, "sim_graph_launch: the layout changed since the graph was created");
    SIM_DEVICE_SCOPE(h, h->device);
    SIM_CUDA_TRY(h, cudaGraphLaunch(g->exec, h->stream));
    h->launches += (uint64_t)g->n_blocks;
    return SIM_OK;
}

int sim_graph_destroy(sim_graph_t *g)
{
    if (!g) return fail(nullptr, SIM_E_INVAL, "sim_graph_destroy: NULL graph");
    DeviceScope dev_scope(g->h->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->d_staged) cudaFree(g->d_staged);
    delete g;
    return SIM_OK;
}

// ---- autotuner: measure candidate widths and arithmetic on the device ----

int sim_autotune(sim_t *h, int n_gates, const sim_gate *gates, int accuracy, sim_plan_opts *best,
                 double *best_ms)
{
    if (!h || !best) return fail(h, SIM_E_INVAL, "sim_autotune: NULL argument");
    state_written(h);
    if (h->store != SIM_STORE_DEVICE || h->s != 0)
        return fail(h, SIM_E_UNSUPPORTED, "sim_autotune: needs a device-resident, unsliced handle");
    if (accuracy != SIM_TUNE_FP32 && accuracy != SIM_TUNE_FP32_EQUIVALENT && accuracy != SIM_TUNE_ANY)
        return fail(h, SIM_E_INVAL, "sim_autotune: accuracy class %d", accuracy);
    std::vector<int> precs = {SIM_FP32};
    if (accuracy != SIM_TUNE_FP32) {
        precs.push_back(SIM_FP16X3);
        precs.push_back(SIM_FP16X3_TMEM);
        precs.push_back(SIM_TF32X3);
    }
    if (accuracy == SIM_TUNE_ANY) {  // the stated-bound modes
        precs.push_back(SIM_TF32);
        precs.push_back(SIM_BF16X3);
    }
    SIM_DEVICE_SCOPE(h, h->device);
    cudaEvent_t e0, e1;
    SIM_CUDA_TRY(h, cudaEventCreate(&e0));
    SIM_CUDA_TRY(h, cudaEventCreate(&e1));
    double best_t = 1e300;
    sim_plan_opts pick{};
    int rc = SIM_OK;
    for (int prec : precs)
        for (int kmax = 3; kmax <= kMaxK && rc == SIM_OK; kmax++) {
            // mma.sync tensor-core paths take blocks of k >= 5, the tcgen05 path k >= 4
            if (prec != SIM_FP32 && kmax < (tmem_mode(prec) ? 4 : 5)) continue;
            sim_plan_opts o{};
            o.kmax = kmax;
            o.precision = prec;
            sim_plan_t *p = nullptr;
            rc = sim_plan_create(h->n, n_gates, gates, &o, &p);
            if (rc != SIM_OK) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == SIM_OK; rep++) {  // first run warms up
                rc = sim_reset(h, 0);
                if (rc == SIM_OK) rc = cudaEventRecord(e0, h->stream) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
                if (rc == SIM_OK) rc = sim_apply_plan(h, p);
                if (rc == SIM_OK) rc = cudaEventRecord(e1, h->stream) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
                if (rc == SIM_OK) rc = cudaEventSynchronize(e1) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
                if (rc == SIM_OK) cudaEventElapsedTime(&ms, e0, e1);
            }
            sim_plan_destroy(p);
            if (rc == SIM_OK && ms < best_t) {
                best_t = ms;
                pick = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SIM_OK) return rc;
    *best = pick;
    if (best_ms) *best_ms = best_t;
    return sim_reset(h, 0);
}

// ---- phases over two alternating sliced sets (Sect. 4) ----

int sim_phases_create(int n_qubits, int n_gates, const sim_gate *gates, const sim_plan_opts *o,
                      int slice_bits, const int *set_a, const int *set_b, sim_phases_t **out)
{
    if (!out) return fail(nullptr, SIM_E_INVAL, "sim_phases_create: out is NULL");
    *out = nullptr;
    if (n_qubits < 2 || n_qubits > kMaxQubits || slice_bits < 1 || slice_bits > 8 ||
        2 * slice_bits >= n_qubits || !set_a || !set_b || (n_gates > 0 && !gates) || n_gates < 0)
        return fail(nullptr, SIM_E_INVAL, "sim_phases_create: bad arguments");
    std::vector<int> which(n_qubits, -1);  // 0: set A, 1: set B
    for (int w = 0; w < 2; w++)
        for (int i = 0; i < slice_bits; i++) {
            const int q = w ? set_b[i] : set_a[i];
            if (q < 0 || q >= n_qubits || which[q] >= 0)
                return fail(nullptr, SIM_E_INVAL, "sim_phases_create: sets must be disjoint qubits");
            which[q] = w;
        }
    double G[32];
    for (int g = 0; g < n_gates; g++) {
        const int d = gate_matrix(gates[g], G);
        if (d == 4 && which[gates[g].q0] >= 0 && which[gates[g].q1] >= 0 &&
            which[gates[g].q0] != which[gates[g].q1])
            return fail(nullptr, SIM_E_NONLOCAL,
                        "sim_phases_create: gate %d couples set A and set B; no phase can apply it", g);
    }
    std::vector<std::pair<int, std::vector<int>>> best, alt;
    const bool ok0 = split_phases(n_qubits, n_gates, gates, which, 0, best),
               ok1 = split_phases(n_qubits, n_gates, gates, which, 1, alt);
    if (!ok0 && !ok1) return fail(nullptr, SIM_E_INVAL, "sim_phases_create: circuit cannot be phased");
    // of the two starting sets, the one with the least phases * 32 + fused blocks (the cost
    // sim_phases_choose_sets uses)
    const int kmax_g = o && o->kmax ? o->kmax : 4, width = search_width(o ? o->search : 0);
    auto cost = [&](const std::vector<std::pair<int, std::vector<int>>> &phs) {
        double blocks = 0;
        for (auto &ph : phs) {
            Grouping gr;
            int bad = 0;
            if (group_gates(n_qubits, gates, ph.second, std::max(2, std::min(kmax_g, kMaxK)), width, gr, &bad))
                return 1e300;
            blocks += (double)gr.qubits.size();
        }
        return 32.0 * (double)phs.size() + blocks;
    };
    if (!ok0 || (ok1 && cost(alt) < cost(best))) best.swap(alt);

    auto *ph = new sim_phases_s();
    ph->n = n_qubits;
    ph->s = slice_bits;
    for (int i = 0; i < slice_bits; i++) {
        ph->set_a[i] = set_a[i];
        ph->set_b[i] = set_b[i];
    }
    for (auto &pr : best) {
        std::vector<sim_gate> sub(pr.second.size());
        for (size_t i = 0; i < pr.second.size(); i++) sub[i] = gates[pr.second[i]];
        sim_plan_t *plan = nullptr;
        const int rc = sim_plan_create(n_qubits, (int)sub.size(), sub.data(), o, &plan);
        if (rc != SIM_OK) {
            sim_phases_destroy(ph);
            return rc;
        }
        ph->set_of.push_back(pr.first);
        ph->plans.push_back(plan);
    }
    *out = ph;
    return SIM_OK;
}

int sim_phases_choose_sets(int n_qubits, int n_gates, const sim_gate *gates, int slice_bits,
                           const sim_plan_opts *o, double phase_weight, int *set_a, int *set_b, int *n_phases,
                           int *n_blocks)
{
    if (n_qubits < 2 || n_qubits > kMaxQubits || slice_bits < 1 || slice_bits > 8 || 2 * slice_bits >= n_qubits ||
        n_gates < 0 || (n_gates > 0 && !gates) || !set_a || !set_b)
        return fail(nullptr, SIM_E_INVAL, "sim_phases_choose_sets: bad arguments");
    const int kmax = o && o->kmax ? o->kmax : 4, width = search_width(o ? o->search : 0);
    if (kmax < 2 || kmax > kMaxK) return fail(nullptr, SIM_E_INVAL, "sim_phases_choose_sets: kmax=%d", kmax);
    if (!(phase_weight > 0.0)) phase_weight = 32.0;
    double G[32];
    for (int g = 0; g < n_gates; g++) {
        const int d = gate_matrix(gates[g], G);
        if (!d || gates[g].q0 < 0 || gates[g].q0 >= n_qubits ||
            (d == 4 && (gates[g].q1 < 0 || gates[g].q1 >= n_qubits || gates[g].q1 == gates[g].q0)))
            return fail(nullptr, SIM_E_INVAL, "sim_phases_choose_sets: gate %d is malformed", g);
    }
    const int s = slice_bits;
    double best_cost = 1e300;
    int best_i = -1, best_j = -1, best_ph = 0, best_bl = 0;
    std::vector<int> which(n_qubits);
    for (int i = 0; i + s <= n_qubits; i++)
        for (int j = i + s; j + s <= n_qubits; j++) {
            std::fill(which.begin(), which.end(), -1);
            for (int t = 0; t < s; t++) {
                which[i + t] = 0;
                which[j + t] = 1;
            }
            bool coupled = false;
            for (int g = 0; g < n_gates && !coupled; g++)
                coupled = gate_matrix(gates[g], G) == 4 && which[gates[g].q0] >= 0 && which[gates[g].q1] >= 0 &&
                          which[gates[g].q0] != which[gates[g].q1];
            if (coupled) continue;
            int cand_ph = 0, cand_bl = 0;
            double cand_cost = 1e300;
            for (int first = 0; first < 2; first++) {
                std::vector<std::pair<int, std::vector<int>>> phases;
                if (!split_phases(n_qubits, n_gates, gates, which, first, phases)) continue;
                int blocks = 0;
                for (auto &ph : phases) {
                    Grouping gr;
                    int bad = 0;
                    if (group_gates(n_qubits, gates, ph.second, kmax, width, gr, &bad))
                        return fail(nullptr, SIM_E_INVAL, "sim_phases_choose_sets: gate %d", bad);
                    blocks += (int)gr.qubits.size();
                }
                const double cost = phase_weight * (double)phases.size() + blocks;
                if (cost < cand_cost) {
                    cand_cost = cost;
                    cand_ph = (int)phases.size();
                    cand_bl = blocks;
                }
            }
            if (cand_cost < best_cost) {
                best_cost = cand_cost;
                best_i = i;
                best_j = j;
                best_ph = cand_ph;
                best_bl = cand_bl;
            }
        }
    if (best_i < 0) return fail(nullptr, SIM_E_INVAL, "sim_phases_choose_sets: no pair of sets can phase the circuit");
    for (int t = 0; t < s; t++) {
        set_a[t] = best_i + t;
        set_b[t] = best_j + t;
    }
    if (n_phases) *n_phases = best_ph;
    if (n_blocks) *n_blocks = best_bl;
    return SIM_OK;
}

int sim_phases_destroy(sim_phases_t *ph)
{
    if (!ph) return fail(nullptr, SIM_E_INVAL, "sim_phases_destroy: NULL");
    for (auto *p : ph->plans) delete p;
    delete ph;
    return SIM_OK;
}

int sim_phases_info(const sim_phases_t *ph, int *n_phases, int *total_blocks)
{
    if (!ph) return fail(nullptr, SIM_E_INVAL, "sim_phases_info: NULL");
    if (n_phases) *n_phases = (int)ph->plans.size();
    if (total_blocks) {
        int t = 0;
        for (auto *p : ph->plans) t += (int)p->blocks.size();
        *total_blocks = t;
    }
    return SIM_OK;
}

int sim_phases_get(const sim_phases_t *ph, int i, int *set, const sim_plan_t **plan)
{
    if (!ph || i < 0 || i >= (int)ph->plans.size())
        return fail(nullptr, SIM_E_INVAL, "sim_phases_get: no phase %d", i);
    if (set) *set = ph->set_of[i];
    if (plan) *plan = ph->plans[i];
    return SIM_OK;
}

int sim_run_phases(sim_t *h, const sim_phases_t *ph)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_run_phases: NULL handle");
    state_written(h);
    if (!ph || ph->n != h->n) return fail(h, SIM_E_INVAL, "sim_run_phases: phases missing or for another n");
    if (h->store == SIM_STORE_HOST) {
        if (ph->s != h->s) return fail(h, SIM_E_INVAL, "sim_run_phases: slice_bits differ");
        for (int i = 0; i < ph->s; i++)
            if (ph->set_a[i] != h->set[0][i] || ph->set_b[i] != h->set[1][i])
                return fail(h, SIM_E_INVAL, "sim_run_phases: sliced sets differ from the handle's");
    }
    for (size_t i = 0; i < ph->plans.size(); i++) {
        if (h->store == SIM_STORE_DEVICE && h->s > 0) {
            // Resident state with sliced top bits (Sect. 4 in device memory): before the phase,
            // move the phase's sliced set into the top slice_bits physical bits, exchanging them
            // with whatever qubits hold those bits (an in-place bit permutation).
            if (ph->s != h->s) return fail(h, SIM_E_INVAL, "sim_run_phases: slice_bits differ");
            const int *X = ph->set_of[i] == 0 ? ph->set_a : ph->set_b;
            std::vector<int> perm(h->n);
            for (int q = 0; q < h->n; q++) perm[q] = h->bit_of[q];
            for (int j = 0; j < ph->s; j++) {
                const int want = h->n - h->s + j, q = X[j];
                if (perm[q] == want) continue;
                int other = -1;
                for (int r = 0; r < h->n; r++)
                    if (perm[r] == want) other = r;
                perm[other] = perm[q];
                perm[q] = want;
            }
            // while the state moves anyway, also move qubits between the low bits where that
            // speeds up this phase's blocks (disjoint swaps: still one permutation pass)
            std::vector<char> used(h->n, 0);
            bool sliced_moved = false;
            for (int q = 0; q < h->n; q++)
                if (perm[q] != h->bit_of[q]) {
                    used[perm[q]] = used[h->bit_of[q]] = 1;
                    sliced_moved = true;
                }
            const std::vector<int> before = perm;
            const double gain = improve_by_disjoint_swaps(ph->plans[i], perm, used, h->n - h->s);
            // without a move of the sliced set the swaps would cost a pass of their own (~3.4 in
            // the estimate's units, a permutation pass on 2^30 amplitudes): keep them only if
            // they save more than that
            if (!sliced_moved && gain > -3.5) perm = before;
            bool moved = false;
            for (int q = 0; q < h->n; q++) moved = moved || perm[q] != h->bit_of[q];
            if (moved) {
                const int rc = sim_permute(h, perm.data());
                if (rc != SIM_OK) return rc;
            }
        }
        const int rc = sim_run_phase(h, ph->set_of[i], ph->plans[i]);
        if (rc != SIM_OK) return rc;
    }
    return SIM_OK;
}

}  // extern "C"
