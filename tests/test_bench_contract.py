"""bench.py on the host: the algorithmic byte model behind the roofline (per tet: corner
ids, B, F(x_t), V_e and material, four incidence entries; per free vertex: x read and
written, z, m, R, g/H written and read, and the cubature record), and the JSON line of
the reference arm (the FP64 oracle on the host cores)."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_byte_model():
    b = _bench()
    assert b.sweep_bytes(0, 1, 4) == 116            # 16 ids + 21 x 4 record + 16 incidence
    assert b.sweep_bytes(1, 0, 4) == 756            # 40 + 36 + 72 + 4 x (4 + 37 x 4)
    assert b.sweep_bytes(634_130, 3_471_360, 4) == 882_080_040   # ten spheres, FP32
    kb = b.kernel_bytes(634_130, 3_471_360, 4, 4)
    assert kb["k_energy"] == 3_471_360 * 100 + 634_130 * 40
    assert kb["k_energy_2"] == 3_471_360 * 100 + 634_130 * 52
    assert kb["k_correct"] == 634_130 * (84 + 4 * 152)


def test_scope_byte_model():
    """The hot-path scope's per-unit figures: 76 B per tet and 756 B per free vertex in FP32
    (743 MB per sweep at 3.47M tets)."""
    b = _bench()
    assert b.scope_sweep_bytes(0, 1, 4) == 76
    assert b.scope_sweep_bytes(1, 0, 4) == 756
    assert abs(b.scope_sweep_bytes(634_130, 3_471_360, 4) - 743e6) < 1e6


def test_makespan():
    b = _bench()
    assert b.makespan([3.0, 1.0, 1.0, 1.0], 2) == 3.0
    assert b.makespan([2.0, 2.0, 2.0], 2) == 4.0
    assert b.makespan([1.0] * 10, 16) == 1.0


def test_reference_arm_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cube", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms/step" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and "sample" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
