"""The benchmark's host side, without a GPU: the reference arm (the FP64 oracle timed on
the host cores) prints one JSON line with the keys and the metric of the GPU arm, ranks
other than 0 print nothing, and the algorithmic per-edge GEMM figures follow from the
layer shapes of the model."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None, timeout=600):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args,
                          capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=e)


def test_reference_arm_line():
    import bench
    r = _run(["--impl", "reference", "--workload", "cubic96", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "cubic96" and d["config"]["atoms"] == 96
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--workload", "cubic96", "--steps", "1", "--warmup", "3"],
             env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_below_three_is_refused():
    r = _run(["--impl", "reference", "--workload", "cubic96", "--steps", "1", "--warmup", "2"])
    assert r.returncode != 0 and "warmup" in r.stderr


def _mac_by_layers(hp):
    """Multiply-adds per edge of one forward pass through the dense layers, written out
    layer by layer from the model's widths (two-body hidden layers after the input layer;
    per interaction layer the env projection D -> (lmax+1) C and the latent MLP over
    [x | scalars])."""
    D = hp["two_body"][-1]
    ldw = (hp["lmax"] + 1) * hp["channels"]
    widths = list(hp["two_body"])
    mac = 0
    for a, b in zip(widths[:-1], widths[1:]):
        mac += a * b
    for _ in range(hp["n_layers"]):
        mac += D * ldw
        fan = D + ldw
        for w in hp["latent"]:
            mac += fan * w
            fan = w
    return mac


@pytest.mark.parametrize("name", ["fm_water", "small", "fm64", "fm256", "fm512"])
def test_gemm_flops_per_edge_from_layer_shapes(name):
    import bench
    import synth
    hp = synth.preset(name)
    # forward products plus the adjoint's input-gradient products of the same shapes
    assert bench.gemm_flops_per_edge(hp) == 2 * 2 * _mac_by_layers(hp)


def test_water_model_figures():
    import bench
    import synth
    hp = synth.preset("fm_water")
    # 64x128 + 128x256 two-body hidden layers; 3 x (256x96 env + 352x256 latent)
    assert _mac_by_layers(hp) == 64 * 128 + 128 * 256 + 3 * (256 * 96 + 352 * 256)
    assert bench.gemm_flops_per_edge(hp) == 1_540_096
    # compulsory bytes of the two paths' GEMM classes, as the roofline uses them
    assert bench.gemm_bytes_per_edge(hp, 1) == 21_848
    assert bench.gemm_bytes_per_edge(hp, 0) == 41_232


def test_method_flops_per_edge_matches_the_model_definition():
    """Matrix-unit work of one E+F per edge as the method defines it, for the config-2
    model: radial input 8x64, two-body 64x128 + 128x256, 3 x (env 256x96 + latent
    352x256), edge-energy 256x128 + 128x1 = 418,432 multiply-adds forward; x2 FLOP, x2
    for the adjoint's input gradients."""
    import bench
    import synth
    hp = synth.preset("fm_water")
    mac = 8 * 64 + 64 * 128 + 128 * 256 + 3 * (256 * 96 + 352 * 256) + 256 * 128 + 128
    assert mac == 418_432
    assert bench.method_flops_per_edge(hp) == 4 * mac == 1_673_728
    # the readout and radial layers are the only difference from the GEMM-shaped work
    assert bench.method_flops_per_edge(hp) - bench.gemm_flops_per_edge(hp) == \
        4 * (8 * 64 + 256 * 128 + 128)
