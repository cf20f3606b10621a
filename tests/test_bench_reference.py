"""Host-side parts of bench.py, CPU only.  The oracle arm (--impl reference) runs on the host CPU
alone: its JSON line carries the keys the benchmark contract asks for, describes its own CPU run,
and prints nothing on a rank other than 0.  The roofline's algorithmic flop counts equal a walk
over each adjoint form's products, and the whole-job value is every rank's units over the slowest
rank's time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3", "--cpu-sample", "20", *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_line_has_the_contract_keys():
    (line,) = run()
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"]
    assert isinstance(cpu["cores"], int) and 1 <= cpu["cores"] <= (os.cpu_count() or 1) + 8
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "transmon_cavity_d40" and line["config"]["sample_slices"] == 20
    assert "flushed" not in line["config"]["l2"]


def test_reference_line_only_on_rank_zero():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _walk_flops(form, d, p, n, S):
    """Algorithmic flops of one slice's exponential adjoint, counted by walking its products:
    a complex (m x k) by (k x q) product is 8 m k q real flops."""
    mm = lambda m, k, q: 8.0 * m * k * q
    if form == 3:                                   # low-rank reverse mode
        f, r = 0.0, S
        for _ in range(n):                          # S R and S^dag L per squaring, rank doubles
            f += mm(d, d, r) + mm(d, d, r)
            r *= 2
        for _ in range(p - 1):                      # W = Z R, X^dag L, L W^dag per Horner step
            f += mm(d, d, r) + mm(d, d, r) + mm(d, r, d)
        return f + mm(d, r, d)                      # L_p R^dag / p
    per_product = {0: 2, 1: 3}[form]                # reverse mode: 2, block recursion: 3
    return per_product * (p - 1 + n) * mm(d, d, d) + mm(d, S, d)   # plus Ubar = G Psi^dag


def _walk_flops_ps(form, d, p, n, S):
    """The same walk for the Paterson-Stockmeyer form (blocks of three terms, top block qt)."""
    mm = lambda m, k, q: 8.0 * m * k * q
    qt = p // 3 - 1 if (p % 3 == 0 and p >= 3) else p // 3
    powers = (2 if p >= 3 else 0) + (2 if p >= 2 else 0)   # Ybar X^dag, X2^dag Ybar; X2bar X^dag, X^dag X2bar
    if form == 0:
        return (2 * n + 2 * qt + powers) * mm(d, d, d) + mm(d, S, d)
    f, r = 0.0, S
    for _ in range(n):
        f += mm(d, d, r) + mm(d, d, r)
        r *= 2
    for _ in range(qt):                             # V = W R, Y^dag L, L V^dag
        f += mm(d, d, r) + mm(d, d, r) + mm(d, r, d)
    if p % 3 == 0 and p >= 3:                       # top block's c L R^dag into Ybar
        f += mm(d, r, d)
    f += 2 * mm(d, r, d)                            # (sum c L) R^dag into Xbar and X2bar
    return f + powers * mm(d, d, d)


def test_roofline_flop_counts():
    b = _bench()
    assert b.expm_flops_per_slice(40, 9, 4) == 12 * 8.0 * 40 ** 3
    for form in (0, 1, 3):
        for d, p, n, S in [(40, 9, 4, 1), (64, 7, 1, 2), (48, 5, 0, 3), (81, 12, 2, 16)]:
            assert b.adj_flops_per_slice(form, d, p, n, S) == _walk_flops(form, d, p, n, S), (form, d, p, n, S)
    assert b.expm_flops_per_slice(40, 14, 2, 1) == 8 * 8.0 * 40 ** 3          # X^2, X^3, 4 chain, 2 squarings
    assert b.expm_flops_per_slice(40, 12, 2, 1) == 7 * 8.0 * 40 ** 3          # 3 | p: the top block folds
    for form in (0, 3):
        for d, p, n, S in [(40, 14, 2, 1), (40, 12, 2, 1), (48, 5, 0, 3), (16, 2, 1, 1), (20, 1, 3, 2)]:
            assert b.adj_flops_per_slice(form, d, p, n, S, 1) == _walk_flops_ps(form, d, p, n, S), (form, d, p, n, S)


def test_job_value_is_all_ranks_over_the_slowest():
    b = _bench()
    assert b.job_value(2000, 1, 2.5) == 2000 / 2.5e-3
    assert b.job_value(2000, 4, 5.0) == 4 * 2000 / 5e-3
    assert b.slowest_rank_ms(3.0, 1, "cpu") == 3.0
