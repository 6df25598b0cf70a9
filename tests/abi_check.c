/*
 * abi_check.c -- a plain C caller of the library, compiled by the tests with gcc against
 * include/sycsim.h, independent of the Python binding.
 *
 *   abi_check layout
 *       prints "struct field offset size" lines for every struct the header declares (and
 *       "struct - sizeof" lines), which the host test compares with the binding's mirrors.
 *   abi_check run <circuit.txt> <out.bin> [kmax precision]
 *       reads a circuit as text ("n_qubits n_gates" then one gate per line: kind q0 q1 theta phi
 *       dplus dminus dminus_off), plans it (sim_plan_create), runs it from |0..0> on a device
 *       state (sim_apply_plan), permutes the qubits to reversed order and back (sim_permute),
 *       reads all amplitudes in logical order as complex128 (sim_amplitudes) and reduces
 *       (sim_reduce); writes norm, 2^n sum p^2, xeb and then the 2^n amplitudes (doubles) to
 *       out.bin.  Exit status 0, or 1 with the library's message on stderr.
 */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include "sycsim.h"

#define FIELD(S, F) printf("%s %s %zu %zu\n", #S, #F, offsetof(S, F), sizeof(((S *)0)->F))
#define SIZE(S) printf("%s - %zu\n", #S, sizeof(S))

static int layout(void)
{
    FIELD(sim_gate, kind);
    FIELD(sim_gate, q0);
    FIELD(sim_gate, q1);
    FIELD(sim_gate, reserved);
    FIELD(sim_gate, theta);
    FIELD(sim_gate, phi);
    FIELD(sim_gate, dplus);
    FIELD(sim_gate, dminus);
    FIELD(sim_gate, dminus_off);
    FIELD(sim_gate, u);
    SIZE(sim_gate);
    FIELD(sim_opts, store);
    FIELD(sim_opts, device);
    FIELD(sim_opts, stream);
    FIELD(sim_opts, ext_state);
    FIELD(sim_opts, ext_bytes);
    FIELD(sim_opts, slots);
    FIELD(sim_opts, set_a);
    FIELD(sim_opts, set_b);
    FIELD(sim_opts, store_device_regions);
    FIELD(sim_opts, reserved);
    SIZE(sim_opts);
    FIELD(sim_plan_opts, kmax);
    FIELD(sim_plan_opts, precision);
    FIELD(sim_plan_opts, search);
    FIELD(sim_plan_opts, reserved);
    SIZE(sim_plan_opts);
    FIELD(srv_opts, device);
    FIELD(srv_opts, slots);
    FIELD(srv_opts, small_n);
    FIELD(srv_opts, max_pack);
    FIELD(srv_opts, kmax);
    FIELD(srv_opts, precision);
    FIELD(srv_opts, hbm_budget);
    FIELD(srv_opts, front_pairs);
    FIELD(srv_opts, max_large);
    FIELD(srv_opts, reserved);
    SIZE(srv_opts);
    FIELD(srv_stats_t, submitted);
    FIELD(srv_stats_t, completed);
    FIELD(srv_stats_t, rejected);
    FIELD(srv_stats_t, in_flight);
    FIELD(srv_stats_t, p50_ms);
    FIELD(srv_stats_t, p99_ms);
    FIELD(srv_stats_t, mean_ms);
    FIELD(srv_stats_t, circuits_per_s);
    FIELD(srv_stats_t, hbm_budget);
    FIELD(srv_stats_t, hbm_used);
    FIELD(srv_stats_t, graph_replays);
    SIZE(srv_stats_t);
    return 0;
}

static int die(const sim_t *h, const char *what, int rc)
{
    fprintf(stderr, "%s: %d: %s\n", what, rc, sim_last_error(h));
    return 1;
}

static int run(const char *circuit_path, const char *out_path, int kmax, int precision)
{
    FILE *f = fopen(circuit_path, "r");
    if (!f) return die(NULL, "open circuit", -1);
    int n = 0, ng = 0;
    if (fscanf(f, "%d %d", &n, &ng) != 2 || n < 1 || n > 30 || ng < 1) {
        fclose(f);
        return die(NULL, "circuit header", -1);
    }
    sim_gate *g = (sim_gate *)calloc((size_t)ng, sizeof(sim_gate));
    for (int i = 0; i < ng; i++) {
        if (fscanf(f, "%d %d %d %lf %lf %lf %lf %lf", &g[i].kind, &g[i].q0, &g[i].q1, &g[i].theta, &g[i].phi,
                   &g[i].dplus, &g[i].dminus, &g[i].dminus_off) != 8) {
            fclose(f);
            free(g);
            return die(NULL, "circuit gate", -1);
        }
    }
    fclose(f);
    sim_plan_opts po = {0};
    po.kmax = kmax;
    po.precision = precision;
    sim_plan_t *p = NULL;
    int rc = sim_plan_create(n, ng, g, &po, &p);
    free(g);
    if (rc) return die(NULL, "sim_plan_create", rc);
    sim_opts o = {0};  /* device 0, own stream, own buffer */
    sim_t *h = NULL;
    if ((rc = sim_create(n, 0, &o, &h))) return die(NULL, "sim_create", rc);
    int *rev = (int *)malloc(sizeof(int) * (size_t)n), *id = (int *)malloc(sizeof(int) * (size_t)n);
    for (int q = 0; q < n; q++) {
        rev[q] = n - 1 - q;
        id[q] = q;
    }
    const size_t amps = (size_t)1 << n;
    double *out = (double *)malloc(sizeof(double) * (3 + 2 * amps));
    if ((rc = sim_apply_plan(h, p))) return die(h, "sim_apply_plan", rc);
    if ((rc = sim_permute(h, rev))) return die(h, "sim_permute", rc);
    if ((rc = sim_permute(h, id))) return die(h, "sim_permute", rc);
    if ((rc = sim_amplitudes(h, 0, amps, out + 3, SIM_C128, 0))) return die(h, "sim_amplitudes", rc);
    if ((rc = sim_reduce(h, out, out + 1, out + 2))) return die(h, "sim_reduce", rc);
    if ((rc = sim_sync(h, 10000))) return die(h, "sim_sync", rc);
    sim_destroy(h);
    sim_plan_destroy(p);
    FILE *w = fopen(out_path, "wb");
    if (!w || fwrite(out, sizeof(double), 3 + 2 * amps, w) != 3 + 2 * amps) return die(NULL, "write", -1);
    fclose(w);
    free(out);
    free(rev);
    free(id);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc >= 2 && argv[1][0] == 'l') return layout();
    if (argc >= 4 && argv[1][0] == 'r')
        return run(argv[2], argv[3], argc >= 5 ? atoi(argv[4]) : 4, argc >= 6 ? atoi(argv[5]) : SIM_FP32);
    fprintf(stderr, "usage: abi_check layout | run circuit.txt out.bin [kmax precision]\n");
    return 2;
}
