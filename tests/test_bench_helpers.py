"""Host-side logic of bench.py and of the seeded inputs (CPU only)."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
from paper_2004_11346_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workload_plan_overrides():
    w = bench.workload("mixed_N1024_F64")
    assert w["plan"] == {"n0": 256, "n_leaf": 256}  # the autotuner's pick for the headline
    w = bench.workload("mixed_N1024_F64", n0=512)
    assert w["plan"] == {"n0": 512, "n_leaf": 256}
    assert "plan" not in bench.workload("fp64_N1024")
    assert bench.config_of(bench.workload("fp64_N1024"), 1)["plan"] == "library defaults"


def test_recorded_tile_matches_the_kernel_source():
    # the bench line's config.tile restates compile-time constants of the
    # tensor-core kernel; read them back from the sources
    import re
    csrc = os.path.join(ROOT, "paper_2004_11346_gb300", "csrc")
    src = open(os.path.join(csrc, "apply_tc.cuh")).read() + open(os.path.join(csrc, "apply_tc.cu")).read()

    def const(name):
        return int(re.search(r"constexpr int %s = (\d+);" % name, src).group(1))

    fields = const("kTcFields")
    assert bench.TC_TILE == {"M_rhs": 4 * fields, "N": const("kTcNT"), "K_chunk": const("kTcKC"),
                             "stages": const("kStages")}
    assert bench.config_of(bench.workload("mixed_N1024_F64"), 1)["tile"] == bench.TC_TILE
    assert "tile" not in bench.config_of(bench.workload("fp64_N1024"), 1)


def test_headline_traffic_scales_from_its_plan_shape(tmp_path, monkeypatch):
    # a capture of a smaller case of the same kernel is scaled by algorithmic bytes
    t = {"mixed_N512_F64_tuned": 300.0, "_algorithmic_mixed_N512_F64_tuned": 200.0, "mixed_N512_F32": 7.0,
         "_algorithmic_mixed_N512_F32": 5.0}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"alt_tc_kernel": t}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    ref = bench.TRAFFIC_REF["mixed_N1024_F64"]
    v, src = bench.traffic_for("alt_tc_kernel", "mixed_N1024_F64", 1000)
    assert ref in src and abs(v - 1000 * t[ref] / t["_algorithmic_" + ref]) < 1e-6
    v, src = bench.traffic_for("alt_tc_kernel", "mixed_N512_F32")
    assert v == t["mixed_N512_F32"]
    assert bench.traffic_for("no_such_kernel", "mixed_N512_F32") == (None, None)


def test_uneven_workload_names():
    assert bench.uneven_sizes("uneven_N128-1024_F256") == ((128, 256, 512, 1024), 256)
    assert bench.uneven_sizes("uneven_N64-64_F8") == ((64,), 8)


def test_uneven_batch_is_seeded_and_consistent():
    sizes = (16, 32, 64)
    per_field, coeffs = inputs.uneven_batch(40, seed=1, sizes=sizes)
    again, coeffs2 = inputs.uneven_batch(40, seed=1, sizes=sizes)
    assert np.array_equal(per_field, again)
    assert set(per_field.tolist()) <= set(sizes) and len(per_field) == 40
    assert sum(c.shape[0] for c in coeffs.values()) == 40
    for N, c in coeffs.items():
        assert c.shape == ((per_field == N).sum(), 4 * N * N, 2)
        assert np.array_equal(c, coeffs2[N])
    # the sizes are the generator's first draw: uniform integers over the size list
    idx = np.random.default_rng(1).integers(0, len(sizes), 40)
    assert np.array_equal(per_field, np.asarray(sizes)[idx])


def test_reference_arm_declines_uneven_batches():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "uneven_N16-32_F4", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_compare_reports_the_paper_ratios(monkeypatch):
    """compare()'s bookkeeping with stand-ins for the GPU parts: the IDBF and
    dense plans' times and build times give the paper's two speedup ratios."""
    class FakeTensor:
        shape = (16,)

        def __getitem__(self, k):
            return self

        def __sub__(self, o):
            return self

        def contiguous(self):
            return self

        def norm(self):
            return 1.0

    class FakeTorch:
        float64 = "f64"

        class cuda:
            @staticmethod
            def empty_cache():
                pass

        @staticmethod
        def empty(*a, **k):
            return FakeTensor()

        @staticmethod
        def empty_like(x):
            return FakeTensor()

    class FakePlan:
        def __init__(self, N, eps, precision=None, flags=0, max_fields=1):
            self.dense = bool(flags & 4)

        def stats(self):
            return {"entries_total": 10, "t_factor_s": 6.0 if self.dense else 2.0}

    class FakeSht:
        Plan = FakePlan

    lib = type("L", (), {"SHT_FP64": 0, "SHT_FLAG_DENSE": 4, "SHT_FLAG_DIRECT": 16})
    # FP64 IDBF, dense stored, dense on the fly (16 fields)
    times = iter([(10.0, 4.0, 6.0), (40.0, 15.0, 25.0), (2000.0, 900.0, 1100.0)])
    monkeypatch.setattr(bench, "time_steps", lambda *a: next(times))
    monkeypatch.setattr(bench, "sht_timings", lambda *a, **k: {})
    args = type("A", (), {"steps": 4})
    out = bench.compare(FakeTorch, FakeSht, lib, {"N": 8, "precision": "fp64"}, None, FakeTensor(), None, args, None)
    assert out["fp64_idbf"]["t_fac_s"] == 2.0 and out["dense_fp64"]["t_mat_s"] == 6.0
    assert out["paper_ratios"] == {"t_dir_over_t_app": 4.0, "t_mat_over_t_fac": 3.0}
    assert out["dense_direct_fp64"]["fields_per_s"] == 8.0 and out["dense_direct_fp64"]["fields"] == 16
