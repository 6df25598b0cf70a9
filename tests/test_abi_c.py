"""The C ABI from C: tests/abi_check.c is compiled with gcc against include/sycsim.h and linked with
the library, with no Python binding in between.

* Host: the struct layouts the C compiler gives the header's types (every field's offset and size,
  every struct's size) equal the binding's mirrors (numpy gate records, ctypes structures), so a
  field added, moved or resized on one side only fails here.
* GPU: the C program reads a per-location detuned 12-qubit circuit as text into sim_gate records,
  plans and runs it, permutes, reads out and reduces through the C ABI; the result must match the
  oracle (||psi - psi_oracle||_2 <= 1e-5, reductions to 1e-6).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import syc_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    p.lib()
    return p


@pytest.fixture(scope="module")
def abi_check(pkg, tmp_path_factory):
    libdir = os.path.join(ROOT, "paper_1910_09534_gb300", "_build")
    exe = str(tmp_path_factory.mktemp("abi") / "abi_check")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_check.c"), "-L", libdir, "-lsycsim", f"-Wl,-rpath,{libdir}",
           "-Wl,--allow-shlib-undefined", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def c_layout(exe):
    out = subprocess.run([exe, "layout"], capture_output=True, text=True, check=True).stdout
    fields, sizes = {}, {}
    for line in out.splitlines():
        s, f, a, *b = line.split()
        if f == "-":
            sizes[s] = int(a)
        else:
            fields[(s, f)] = (int(a), int(b[0]))
    return fields, sizes


def test_struct_layouts_match_the_binding(pkg, abi_check):
    fields, sizes = c_layout(abi_check)
    # gate records: numpy structured dtype
    dt = pkg._native.GATE_DTYPE
    for name in dt.names:
        off = dt.fields[name][1]
        assert fields[("sim_gate", name)] == (off, dt.fields[name][0].itemsize), name
    assert sizes["sim_gate"] == dt.itemsize
    assert {f for (s, f) in fields if s == "sim_gate"} == set(dt.names)
    # option and statistics structs: ctypes mirrors
    for cname, py in (("sim_opts", pkg._native.SimOpts), ("sim_plan_opts", pkg._native.PlanOpts),
                      ("srv_opts", pkg._native.SrvOpts), ("srv_stats_t", pkg._native.SrvStats)):
        names = [f for f, _ in py._fields_]
        assert {f for (s, f) in fields if s == cname} == set(names), cname
        for f in names:
            d = getattr(py, f)
            assert fields[(cname, f)] == (d.offset, d.size), (cname, f)
        assert sizes[cname] == ctypes.sizeof(py), cname


def write_circuit(path, circ):
    with open(path, "w") as f:
        f.write(f"{circ.n_qubits} {circ.n_gates}\n")
        for g in circ.gates:
            g = tuple(g) + (0.0,) * (8 - len(g))
            f.write("%d %d %d %.17g %.17g %.17g %.17g %.17g\n" % g)


@pytest.mark.gpu
@pytest.mark.parametrize("kmax,prec_name", [(4, "SIM_FP32"), (5, "SIM_FP16X3_TMEM")])
def test_c_program_runs_a_circuit_like_the_oracle(pkg, oracle_mod, abi_check, tmp_path, kmax, prec_name):
    circ = si.detuned_sycamore_circuit(si.Grid(3, 4), cycles=8, seed=77)
    cpath, opath = str(tmp_path / "circ.txt"), str(tmp_path / "out.bin")
    write_circuit(cpath, circ)
    r = subprocess.run([abi_check, "run", cpath, opath, str(kmax), str(getattr(pkg, prec_name))],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(opath, dtype=np.float64)
    norm, s2, xeb = raw[:3]
    got = raw[3:].view(np.complex128)
    want = oracle_mod.run_circuit(circ)
    assert got.size == want.size
    assert np.linalg.norm(got - want) <= 1e-5
    onorm, os2, oxeb = oracle_mod.reduce(want)
    assert abs(norm - onorm) <= 1e-6 and abs(s2 - os2) <= 1e-5 * os2 and abs(xeb - oxeb) <= 1e-5 * os2
