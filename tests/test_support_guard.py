"""The benchmark's support leg records a failing workload instead of ending the
run (CPU only: no workload is launched)."""

from paper_2110_01614_gb300 import support_bench


def test_guarded_records_the_error_and_wall_time():
    def boom():
        raise RuntimeError("no device")
    r = support_bench.guarded(boom)
    assert r["error"] == "RuntimeError: no device"
    assert r["wall_s"] >= 0.0


def test_guarded_passes_a_record_through():
    r = support_bench.guarded(lambda: {"ms": 1.5})
    assert r["ms"] == 1.5 and "error" not in r and r["wall_s"] >= 0.0


def test_support_line_keeps_going_after_a_failure(monkeypatch):
    calls = []

    def fail(*a, **k):
        calls.append("fail")
        raise ValueError("bad shape")

    def ok(name):
        def f(*a, **k):
            calls.append(name)
            return {"ok": name}
        return f

    for name in ("bench_grouped", "bench_tiny", "bench_penalty", "bench_fit_pool", "bench_kernels"):
        monkeypatch.setattr(support_bench, name, ok(name))
    monkeypatch.setattr(support_bench, "bench_fit512", fail)
    monkeypatch.setattr(support_bench, "fit_body", lambda: ("blob", {}))
    monkeypatch.setattr(support_bench, "bench_cloth_fitted", lambda fitted: {"ok": "cloth"})
    monkeypatch.setattr(support_bench, "bench_voxel", fail)
    out = support_bench.bench_line_support()
    assert out["fit512_bf16"]["error"] == "ValueError: bad shape"
    assert out["voxel"]["error"] == "ValueError: bad shape"
    assert out["kernels"]["ok"] == "bench_kernels" and out["cloth"]["ok"] == "cloth"
    assert set(out) == {"grouped", "tiny", "penalty_gradient", "fit_width64_fp32", "fit512_bf16",
                        "kernels", "cloth", "voxel"}
