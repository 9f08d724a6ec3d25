"""The committed ncu summaries keep the fields bench.py reads in a form it
can parse: a 16-digit hex source hash and whole byte counts (a note after a
number would silently turn the bench line's traffic figure into null)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fields(path):
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                out[k.strip()] = v.strip().strip("`")
    return out


def test_profile_fields_parse():
    seen = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        f = _fields(path)
        if "dram_bytes_per_launch" not in f:
            continue
        seen += 1
        assert re.fullmatch(r"[0-9a-f]{16}", f.get("source_sha256", "")), path
        assert int(f["dram_bytes_per_launch"]) > 0, path
        if "algorithmic_bytes_per_launch" in f:
            assert int(f["algorithmic_bytes_per_launch"]) > 0, path
    assert seen >= 2


def test_bench_reads_the_traffic_figures():
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class W:
        name = "forward_512x512x256_density"

    for kernel, sources in (("step_kernel_forward", bench.KERNEL_SOURCES),
                            ("cpml_step", bench.PML_SOURCES)):
        path = os.path.join(ROOT, "profiles", f"{kernel}_{W.name}.md")
        f = _fields(path)
        got = bench.kernel_traffic(W(), kernel, sources)
        if f["source_sha256"] == bench.kernel_source_hash(sources):
            assert got == int(f["dram_bytes_per_launch"])
        else:  # the kernel changed after the capture: no figure
            assert got is None


def test_algorithmic_bytes_agree_with_the_bench():
    """The algorithmic bytes a profile quotes are the ones bench.py divides by
    the step time: 20 B per padded point for the headline step with density,
    and that plus 16 B per layer point and axis for the CPML step."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2502_12350_gb300 import synth

    w = synth.forward_density(nt=1)
    pts = (w.nx + 2 * w.border) * (w.ny + 2 * w.border) * (w.nz + 2 * w.border)
    head = _fields(os.path.join(ROOT, "profiles",
                                "step_kernel_forward_forward_512x512x256_density.md"))
    assert int(head["algorithmic_bytes_per_launch"]) == 20 * pts
    pml = _fields(os.path.join(ROOT, "profiles", "cpml_step_forward_512x512x256_density.md"))
    assert int(pml["algorithmic_bytes_per_launch"]) == bench.pml_bytes_per_step(w)
