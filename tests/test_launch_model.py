"""The kernel-launch count `bench.py` reports (`gpu_launches`) follows a
per-call model of the launches each public call issues; this pins it to the
count taken from the launch list of one training step of the 256^3-sample
workload (Chebyshev form, 4x128 network, training loss): 90 launches."""
import pytest

torch = pytest.importorskip("torch")


def test_launches_per_step_matches_the_launch_list():
    from paper_2605_29097_gb300 import pipeline as PL
    ch = PL.LAUNCHES_CHEBYSHEV
    n = PL.LAUNCHES["sample"] + 3 * PL.LAUNCHES["fields"] + PL.LAUNCHES["blend"] + PL.LAUNCHES["blend_backward"]
    n += ch["render"] + ch["filter"] + ch["filter_backward"] + ch["render_backward"]
    n += PL.fields_backward_launches(4)
    assert n == 90
