"""Host-side helpers of bench.py: the kernel-source hash that ties a
committed ncu summary to the sources it was taken on, the lookup of the
profiled DRAM traffic, and the autotuner summary in the JSON line."""
import os
import shutil

import bench


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_1411_2181_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench.STEP_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1411_2181_gb300", "csrc", fn), csrc / fn)
    (root / "profiles").mkdir()
    return root, csrc


def test_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    root, csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash() and len(h0) == 16
    f = csrc / "lbfe_fused.cu"
    src = f.read_text()
    f.write_text("// a new comment line\n" + src.replace("namespace lbfe {", "namespace lbfe {  /* note */", 1))
    assert bench.kernel_source_hash() == h0
    f.write_text(src + "\nstatic int extra_symbol = 0;\n")
    assert bench.kernel_source_hash() != h0


def test_profiled_traffic_requires_matching_hash(tmp_path, monkeypatch):
    root, _ = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.kernel_source_hash()
    md = root / "profiles" / "step_demo_fp32.md"
    md.write_text(f"kernel source hash: `{h}`\n| traffic | **dram bytes per lattice update: 329.5** |\n")
    val, fn = bench.profiled_traffic("demo", 0)
    assert val == 329.5 and fn == str(md)
    md.write_text("kernel source hash: `0123456789abcdef`\n| dram bytes per lattice update: 329.5 |\n")
    assert bench.profiled_traffic("demo", 0)[0] is None
    assert bench.profiled_traffic("missing", 0) == (None, None)


def test_committed_profiles_name_a_hash_and_a_traffic_figure():
    for prec in ("fp32", "fp16"):
        fn = os.path.join(bench.ROOT, "profiles", f"step_matrix_ve_192x96x80_{prec}.md")
        txt = open(fn).read()
        assert "kernel source hash:" in txt and "dram bytes per lattice update:" in txt


def test_autotune_summary_keeps_the_fastest_chunk_per_shape():
    shape = {"trials": [[0, 8, 0, 0.16], [0, 8, 40, 0.142], [0, 12, 0, 0.141], [0, 12, 27, 0.15],
                        [1, 16, 0, 0.2]]}
    s = bench.autotune_summary(shape)["best_ms_per_step"]
    assert s == {"cell_32x8": 0.142, "cell_32x12": 0.141, "pair_32x16": 0.2}
    assert bench.autotune_summary(None) is None
