"""The oracle's pins have teeth: each plausible mistake below, planted in a copy of
oracle.c compiled on the CPU, makes at least one pin in test_oracle_march.py,
test_oracle_render.py or test_oracle_fused.py fail. (Mistakes are planted only in
the oracle, never in the CUDA path, and only on the CPU.)
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = [
    ("cell index x/z transposed", "+ ix) * res[1];", "+ iz) * res[1];"),
    ("lookup at interval start, not midpoint", "float mid = (ts + te) * 0.5f;", "float mid = ts;"),
    ("slab exit taken as max", "if (tmax < t_out) t_out = tmax;", "if (tmax > t_out) t_out = tmax;"),
    ("lattice end off by one", "tn = near + (float)(k + 1) * dt_min;", "tn = near + (float)(k + 2) * dt_min;"),
    ("far not clipped", "float te = tn < far ? tn : far;", "float te = tn;"),
    ("time bin rounded, not floored", "return (int)v;", "return (int)(v + 0.5f);"),
    ("cascade level scale off by one", "ldexpf(1.0f, l)", "ldexpf(1.0f, l + 1)"),
    ("cone step not clamped below", "if (dt < dt_min) dt = dt_min;", ""),
    ("Eq. 1 alpha with the printed (dropped) minus sign", "double ai = 1.0 - exp(-tau);", "double ai = 1.0 - exp(tau);"),
    ("inclusive transmittance", "double Ti = exp(-o_acc);", "double Ti = exp(-(o_acc + tau));"),
    ("depth at interval start", "double tmid = ((double)t_starts[off + i] + (double)t_ends[off + i]) * 0.5;",
     "double tmid = (double)t_starts[off + i];"),
    ("gradient uses T_k for T_{k+1}", "double dtau = ak * Tn[k] - suffix;", "double dtau = ak * T[k] - suffix;"),
    ("gradient suffix inclusive", "double dtau = ak * Tn[k] - suffix;", "double dtau = ak * Tn[k] - (suffix + ak * w[k]);"),
    ("gradient missing delta", "d_sigmas[off + k] = delta * dtau;", "d_sigmas[off + k] = dtau;"),
    ("gradient drops the depth term", "+ ga + gd * tmid;", "+ ga;"),
    ("prune on inclusive optical depth", "if (use_t && !(o_acc <= thr_o)) k = 0;",
     "if (use_t && !(o_acc + tau <= thr_o)) k = 0;"),
    ("prune alpha on sigma, not sigma*delta", "float tau = sigmas[i] * delta;", "float tau = sigmas[i];"),
    ("grid decay dropped", "ema[c] = (float)((double)decay * (double)ema[c]);", "ema[c] = ema[c];"),
    ("grid NaN not ignored", "if (v == v && v > ema[c]) ema[c] = v;", "if (!(v <= ema[c])) ema[c] = v;"),
    ("contraction without the 1/|x| factor", "float sc = (2.0f - 1.0f / n) / n;", "float sc = (2.0f - 1.0f / n);"),
    ("contracted grid spans [-1, 1]", "u[a] = (xn[a] + 2.0f) * ((float)res[a] * 0.25f);",
     "u[a] = (xn[a] + 1.0f) * ((float)res[a] * 0.5f);"),
    ("weights gradient uses T_k for T_{k+1}", "d_sigmas[off + k] = delta * (gk * Tn[k] - suffix);",
     "d_sigmas[off + k] = delta * (gk * T[k] - suffix);"),
    ("weights gradient suffix without the weights", "suffix += gk * w[k];", "suffix += gk;"),
    ("accumulate gradient of values without the weight", "d_values[i * n_channels + c] = weights[i] * g;",
     "d_values[i * n_channels + c] = g;"),
    ("accumulate gradient of weights ignores values", "dw += values ? g * (double)values[i * n_channels + c] : g;",
     "dw += g;"),
    ("density lerp along y uses the z fraction", "float c0 = or_lerp(c00, c01, f[1]);",
     "float c0 = or_lerp(c00, c01, f[2]);"),
    ("density vertices x-fastest", "grid[((int64_t)(i[0] + dx) * G[1] + (i[1] + dy)) * G[2] + (i[2] + dz)]",
     "grid[((int64_t)(i[2] + dz) * G[1] + (i[1] + dy)) * G[0] + (i[0] + dx)]"),
    ("density scale by G, not G - 1", "float s = (float)(G[a] - 1) / (box[3 + a] - box[a]);",
     "float s = (float)G[a] / (box[3 + a] - box[a]);"),
    ("density far face outside", "if (!(u >= 0.0f && u <= (float)(G[a] - 1))) return 0.0f;",
     "if (!(u >= 0.0f && u < (float)(G[a] - 1))) return 0.0f;"),
    ("fused density at interval start", "float mid = (ts[i] + te[i]) * 0.5f;", "float mid = ts[i];"),
    ("fused sigma output not compacted", "if (j < capacity) sigmas_out[j] = sg[i];",
     "if (j < capacity) sigmas_out[j] = sg[j];"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site not found: " + old
    mutated = src.replace(old, new)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
                           "-o", str(lib), str(cpath), "-lm"])
    env = dict(os.environ, NACC_ORACLE_LIB_OVERRIDE=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_march.py"), os.path.join(HERE, "test_oracle_render.py"),
                        os.path.join(HERE, "test_oracle_fused.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant '%s' survived every pin:\n%s" % (name, r.stdout[-2000:])
