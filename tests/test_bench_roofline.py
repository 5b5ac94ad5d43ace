"""bench.py's roofline inputs on CPU: the algorithmic bytes of each pack-reading launch
(the per-node matrix entries of the reduced backward sweep, Alg. 1 in the Lambda r
form, plus each launch's node vectors) and the rule that a recorded DRAM traffic
figure is used only while the kernel source it was measured on is unchanged."""
import hashlib
import json
import os

import bench

N, NX, NU, NV = 2081, 63, 114, 97  # the 2081-node Barcelona-shaped tree
NK = NX + NU


def test_stage_bytes_per_node_match_the_matrix_entries():
    # [Bbar; L]' y reads (n_x + n_u) x n_v entries; Lambda r and [Bbar; L] delta read
    # n_v x n_v and (n_x + n_u) x n_v: 17 169 + 9 409 + 17 169 = 43 747 per node-iteration
    assert NK * NV == 17169 and NV * NV == 9409
    gt = bench.stage_bytes("node_mv_gt", N, NX, NU, NV, 1, False)
    dh = bench.stage_bytes("node_mv_dh", N, NX, NU, NV, 1, False)
    chain = bench.stage_bytes("apg_iter_gt", N, NX, NU, NV, 1, False)
    assert gt == N * 4 * (NK * NV + NK + NV)
    assert dh == N * 4 * (NK * NV + NV * NV + NV + NK)
    assert chain == N * 4 * (NK * NV + NK + NX + 2 * NV)
    assert round(gt / 1e6, 1) == 145.2 and round(dh / 1e6, 1) == 223.5 and round(chain / 1e6, 1) == 146.5
    # bfloat16 packs halve the matrix bytes, not the float32 vectors
    assert bench.stage_bytes("node_mv_dh", N, NX, NU, NV, 2, False) == N * (2 * (NK * NV + NV * NV) + 4 * (NV + NK))
    # a shared pack leaves only the vectors
    assert bench.stage_bytes("node_mv_dh", N, NX, NU, NV, 1, True) == N * 4 * (NV + NK)
    # kernels without a pack have no byte model
    assert bench.stage_bytes("prox_node", N, NX, NU, NV, 1, False) is None
    # the fused backward pass reads each pack once: [Bbar; L] and Lambda, w and beta in, h out,
    # s and r published
    fused = bench.stage_bytes("apg_iter_bwd", N, NX, NU, NV, 1, False)
    assert fused == N * 4 * (NK * NV + NV * NV + 2 * NK + NX + 2 * NV)
    assert round(fused / 1e6, 1) == 226.3


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "paper_1604_01074_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "kernels.cu").write_bytes(b"// kernels v1\n")
    sha = hashlib.sha256(b"// kernels v1\n").hexdigest()[:16]
    rec = {"kernel_sha256_16": sha, "fp32_node_mv_dh": {"dram_bytes_per_launch": 230227712}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.recorded_traffic("fp32_node_mv_dh") == 230227712
    assert bench.recorded_traffic("fp32_apg_iter_gt") is None  # not captured
    (src / "kernels.cu").write_bytes(b"// kernels v2\n")  # changed since the capture
    assert bench.recorded_traffic("fp32_node_mv_dh") is None


def test_committed_traffic_matches_the_committed_kernels():
    """profiles/traffic.json names the source it was captured on; while that is the
    committed kernels.cu, its figures are within a few percent of the algorithmic bytes."""
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = json.load(open(os.path.join(here, "profiles", "traffic.json")))
    src = open(os.path.join(here, "paper_1604_01074_gb300", "csrc", "kernels.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != rec["kernel_sha256_16"]:
        return  # kernels changed since the capture: bench.py reports traffic null
    for key, val in rec.items():
        if not isinstance(val, dict):
            continue
        prec, rest = key.split("_", 1)
        stage, n = rest.rsplit("_", 1)
        ratio = val["dram_bytes_per_launch"] / bench.stage_bytes(stage, int(n), NX, NU, NV,
                                                                 {"fp32": 1, "bf16": 2}[prec], False)
        assert 1.0 <= ratio <= 1.08, (key, ratio)
