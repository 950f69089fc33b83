"""Host-side arithmetic of the benchmark line (CPU only).

The roofline numerator is the algorithmic contraction work per (k, q) pair, 8 nw^2 (nRe + 3nat nRp)
flops (one complex multiply-add = 8 flops) for the Wannier-to-Bloch sums of H(k+q) and of
g(k,q) U_k; the configurations' models give the figures the line reports.  The DRAM traffic of
the dominant kernel is read from a committed ncu summary only while the kernel source still has
the hash recorded beside the figure.
"""
import hashlib

import bench
import workloads as W


def test_algorithmic_flops_per_pair_of_the_configurations():
    for name, want in (("fcc_nw4", 69120), ("diamond_nw8", 892416), ("hex_nw5", 610000)):
        m = W.make_workload(name, nq_sub=1).model
        h, g, _ = bench.flops_per_pair(m)
        assert h + g == want, name
        # the H(k+q) part alone: 8 nRe nw^2
        assert h == 8 * m.nw ** 2 * len(m.Re)
    m = W.make_workload("diamond_nw8", nq_sub=1).model
    assert bench.flops_per_pair(m)[0] == 127488


def test_profiled_traffic_follows_the_source_hash(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "k.md"
    prof.write_text(f"# summary\n\n`traffic_per_pair bf16x3 1234.5 source-sha256 {sha}`\n")
    v, why = bench.profiled(str(prof), str(src), "traffic_per_pair", "bf16x3")
    assert v == 1234.5 and "ncu" in why
    assert bench.profiled(str(prof), str(src), "traffic_per_pair", "tf32x3") == (None, "no ncu capture recorded")
    src.write_text("__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench.profiled(str(prof), str(src), "traffic_per_pair", "bf16x3") == (None, "kernel changed since the ncu capture")
    assert bench.profiled(str(tmp_path / "none.md"), str(src), "traffic_per_pair", "bf16x3")[0] is None

