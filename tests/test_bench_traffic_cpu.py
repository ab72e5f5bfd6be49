"""The roofline's DRAM traffic comes from a committed ncu summary only while
that summary still describes the kernel the bench runs: same kernel source
(hash of the file), same leaf size, same k-NN launch shape; otherwise the
bench reports none.  Checked on a temporary tree, without a GPU."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def write_tree(tmp, src_text, sha=None, leaf=16, shape="128x32", dram=123456789):
    os.makedirs(os.path.join(tmp, "profiles"), exist_ok=True)
    os.makedirs(os.path.join(tmp, "k"), exist_ok=True)
    with open(os.path.join(tmp, "k", "knn.cu"), "w") as fh:
        fh.write(src_text)
    if sha is None:
        sha = hashlib.sha256(src_text.encode()).hexdigest()[:16]
    with open(os.path.join(tmp, "profiles", "k_knn_3d_10M.md"), "w") as fh:
        fh.write("# summary\n\nkernel_source: k/knn.cu\nsource_sha256_16: %s\n"
                 "dram_bytes_per_launch: %d\nleaf_size: %d\nknn_shape: %s\n\n| metric | value |\n"
                 % (sha, dram, leaf, shape))


@pytest.fixture
def tree(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return str(tmp_path)


def test_matching_summary_gives_its_bytes(tree):
    write_tree(tree, "kernel A\n")
    assert bench.recorded_traffic("k_knn", 16, "128x32") == 123456789


def test_changed_source_gives_none(tree):
    write_tree(tree, "kernel A\n")
    with open(os.path.join(tree, "k", "knn.cu"), "a") as fh:
        fh.write("// edited\n")
    assert bench.recorded_traffic("k_knn", 16, "128x32") is None


def test_other_leaf_or_shape_gives_none(tree):
    write_tree(tree, "kernel A\n", leaf=16, shape="128x32")
    assert bench.recorded_traffic("k_knn", 8, "128x32") is None
    assert bench.recorded_traffic("k_knn", 16, "256x32") is None


def test_missing_summary_or_source_gives_none(tree):
    assert bench.recorded_traffic("k_knn", 16, "128x32") is None
    write_tree(tree, "kernel A\n")
    os.remove(os.path.join(tree, "k", "knn.cu"))
    assert bench.recorded_traffic("k_knn", 16, "128x32") is None


def test_committed_summary_is_well_formed():
    """The committed k-NN summary names a source file that exists and carries
    every field the bench reads."""
    text = open(os.path.join(ROOT, "profiles", "k_knn_3d_10M.md")).read()
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("kernel_source:", "source_sha256_16:", "dram_bytes_per_launch:",
                                      "leaf_size:", "knn_shape:")))
    assert set(fields) == {"kernel_source", "source_sha256_16", "dram_bytes_per_launch", "leaf_size", "knn_shape"}
    assert os.path.exists(os.path.join(ROOT, fields["kernel_source"].strip()))
    assert int(fields["dram_bytes_per_launch"]) > 0
    assert len(fields["source_sha256_16"].strip()) == 16
