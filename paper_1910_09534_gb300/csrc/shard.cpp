// shard.cpp -- the exchange schedule of a state sharded over global qubits (Sect. 4: the state is
// split over 2^g memories by g "global" qubits, gates act on the local ones, and between phases
// the memory layout is reorganised by an all-to-all so that other qubits become local; the
// Appendix's `all2all` steps).  Host only: it says which local permutation to apply and how the
// all-to-all moves the chunks; the caller's collective library moves the data.
//
// Layout of a sharded state of n qubits over 2^g ranks: position p < n - g is bit p of a rank's
// local index, position n - g + j is bit j of the rank.  An exchange that makes the set X global:
// the m qubits of X that are local (O) trade places with the m global qubits not in X (I).  Each
// rank first permutes its local state so that O[i] sits at local position n - g - m + i (the top
// m local bits), where R[i], the rank bit of I[i], ascending in i, is the bit O[i] will occupy.
// The local state is then 2^m contiguous chunks by the value c of those m bits; chunk c goes to
// the rank whose bits R hold c (the other rank bits equal the sender's), and the chunk received
// from rank s lands at the position given by s's bits R.  Afterwards O[i] is rank bit R[i] and
// I[i] is local position n - g - m + i.  With R ascending, both the destinations of the chunks and
// the sources of the received ones are in rank order, so one all_to_all with per-rank split
// sizes (2^(n-g-m) amplitudes for the 2^m partners, 0 for everyone else) performs it.
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace sycsim;

extern "C" int sim_shard_exchange_plan(int n_qubits, int global_bits, const int *bit_of, const int *next_global,
                                       int *local_perm, int *bit_of_after, uint64_t *chunk_mask)
{
    const int n = n_qubits, g = global_bits;
    if (n < 1 || n > kMaxQubits || g < 0 || g >= n || 2 * g > n)
        return fail(nullptr, SIM_E_INVAL, "sim_shard_exchange_plan: n=%d, g=%d (need 0 <= g, 2g <= n)", n, g);
    if (!bit_of || (g > 0 && !next_global) || !local_perm || !bit_of_after)
        return fail(nullptr, SIM_E_INVAL, "sim_shard_exchange_plan: NULL argument");
    std::vector<int> q_at(n, -1);
    for (int q = 0; q < n; q++) {
        if (bit_of[q] < 0 || bit_of[q] >= n || q_at[bit_of[q]] >= 0)
            return fail(nullptr, SIM_E_INVAL, "sim_shard_exchange_plan: bit_of is not a bijection on 0..%d", n - 1);
        q_at[bit_of[q]] = q;
    }
    std::vector<char> want(n, 0);
    for (int j = 0; j < g; j++) {
        const int q = next_global[j];
        if (q < 0 || q >= n || want[q])
            return fail(nullptr, SIM_E_INVAL, "sim_shard_exchange_plan: next_global[%d]=%d repeated or out of range", j, q);
        want[q] = 1;
    }
    const int L = n - g;
    // I: global qubits leaving (their rank bits R, ascending); O: local qubits entering
    std::vector<int> R, I, O;
    for (int j = 0; j < g; j++) {
        const int q = q_at[L + j];
        if (!want[q]) {
            R.push_back(j);
            I.push_back(q);
        }
    }
    for (int j = 0; j < g; j++)
        if (bit_of[next_global[j]] < L) O.push_back(next_global[j]);
    const int m = (int)O.size();  // == I.size()
    // local permutation: O[i] to local position L - m + i, by successive transpositions
    std::vector<int> at(q_at.begin(), q_at.begin() + L);  // local position -> qubit
    std::vector<int> pos(n);
    for (int q = 0; q < n; q++) pos[q] = bit_of[q];
    for (int i = 0; i < m; i++) {
        const int t = L - m + i, p = pos[O[i]];
        if (p == t) continue;
        const int other = at[t];
        std::swap(at[p], at[t]);
        pos[O[i]] = t;
        pos[other] = p;
    }
    for (int p = 0; p < L; p++) local_perm[p] = pos[q_at[p]];
    // after the all-to-all: O[i] at rank bit R[i], I[i] at local position L - m + i
    for (int q = 0; q < n; q++) bit_of_after[q] = pos[q];
    for (int i = 0; i < m; i++) {
        bit_of_after[O[i]] = L + R[i];
        bit_of_after[I[i]] = L - m + i;
    }
    if (chunk_mask) {
        uint64_t mask = 0;
        for (int r : R) mask |= 1ull << r;
        *chunk_mask = mask;
    }
    return m;
}
