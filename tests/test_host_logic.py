"""Host-side logic of the bench and the autotuner, on CPU: the autotune cache key, the 'traffic:' lines of the
ncu summaries (read only while the kernel source keeps the hash they were taken on), and the algorithmic bytes
of the view conversions."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_autotune_cache_key_buckets_occupancy():
    from paper_2502_16517_gb300 import autotune, sph
    k = autotune.cache_key("GB300", sph.SPH_F64, "grid", 14.9)
    assert k == "GB300|f64|grid|ppc2^4"
    assert autotune.cache_key("GB300", sph.SPH_F32, "patches", 132.0) == "GB300|f32|patches|ppc2^7"
    assert autotune.cache_key("GB300", sph.SPH_F32, "grid", 0.2).endswith("ppc2^0")  # below one particle per cell
    # one bucket per power of two, rounded in log2: 12 and 16 share one, 11 falls in the one below
    assert autotune.cache_key("GB300", sph.SPH_F64, "grid", 12.0) == autotune.cache_key("GB300", 0, "grid", 16.0)
    assert autotune.cache_key("GB300", sph.SPH_F64, "grid", 11.0) != autotune.cache_key("GB300", 0, "grid", 16.0)


def _profile(tmp_path, src_bytes, sha, kernel="k_x<A>", nbytes=123):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "src").mkdir()
    (tmp_path / "src" / "k.cu").write_bytes(src_bytes)
    (tmp_path / "profiles" / "k_x.md").write_text(
        "# summary\n\n```\n"
        f"traffic: kernel={kernel} bytes_per_launch={nbytes} source=src/k.cu sha256={sha}\n```\n")


def test_profiled_traffic_reads_matching_hash(tmp_path):
    src = b"__global__ void k() {}\n"
    _profile(tmp_path, src, hashlib.sha256(src).hexdigest())
    t, where = bench.profiled_traffic("k_x<A>", root=str(tmp_path))
    assert t == 123 and where == os.path.join("profiles", "k_x.md")


def test_profiled_traffic_is_none_once_the_source_changed(tmp_path):
    _profile(tmp_path, b"__global__ void k() { /* edited */ }\n", hashlib.sha256(b"old").hexdigest())
    t, why = bench.profiled_traffic("k_x<A>", root=str(tmp_path))
    assert t is None and "changed" in why


def test_profiled_traffic_unknown_kernel(tmp_path):
    src = b"x"
    _profile(tmp_path, src, hashlib.sha256(src).hexdigest())
    t, why = bench.profiled_traffic("k_other<B>", root=str(tmp_path))
    assert t is None and "no ncu capture" in why


def test_committed_traffic_lines_name_existing_sources():
    # every committed 'traffic:' line names a source in the repository and a 64-hex-digit hash
    found = 0
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        with open(os.path.join(ROOT, "profiles", name), encoding="utf-8") as fh:
            for line in fh:
                if line.startswith("traffic: "):
                    kv = dict(tok.split("=", 1) for tok in line.split()[1:])
                    assert os.path.isfile(os.path.join(ROOT, kv["source"]))
                    assert len(kv["sha256"]) == 64 and int(kv["bytes_per_launch"]) > 0
                    found += 1
    assert found >= 2


@pytest.mark.parametrize("prec,union,per_particle", [
    (0, True, (9 * 8 + 9 * 8 + 4, 7 * 8 + 7 * 8 + 4)),           # {x,v,m,h,u} in, {rho,P,cs,a,du/dt} out
    (1, True, (9 * 8 + 9 * 4 + 4 + 4, 7 * 8 + 7 * 4 + 4)),       # FP32 SoA side, + the slot's cell for positions
    (0, False, ((6 + 11) * 16 + 8, (3 + 4) * 16 + 8)),            # one view per loop, each with its perm read
])
def test_conversion_bytes(prec, union, per_particle):
    g, s = bench.conversion_bytes(prec, 1000, union)
    assert (g, s) == (1000 * per_particle[0], 1000 * per_particle[1])


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 0.5) == 8000.0
