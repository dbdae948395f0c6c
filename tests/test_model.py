"""The byte / flop model reproduces the paper's worked example (golden file
tests/golden/paper_e1.txt, Sec. 2 after Eq. 5)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_e1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                vals[k] = [float(x) for x in v]
    return vals


def _model():
    # load by path: the model is plain host bookkeeping and must not need
    # the CUDA library to be importable
    import importlib.util
    p = os.path.join(os.path.dirname(HERE), "paper_1111_0125_gb300", "model.py")
    spec = importlib.util.spec_from_file_location("stg_model", p)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_paper_worked_example():
    g, m = _golden(), _model()
    assert m.paper_bytes_per_site("f64", 18) == g["bytes_per_site"][0]
    assert m.FLOPS_PER_SITE == g["flops_per_site"][0]
    dims = tuple(int(v) for v in g["lattice"])
    flops, nbytes = m.dslash_totals(dims, "f64", 18)
    assert m.even_sites(dims) == 1053696
    assert flops == 1053696 * 576 and nbytes == 1053696 * 1584
    # printed "0.6 billion" flops: 0.607e9 rounds to 0.6
    assert round(flops / 1e9, 1) == g["gflop_even_sites"][0]
    # printed "1.6 giga bytes": 1.669e9 B, i.e. 1.55 GiB (rounds to 1.6) or
    # 1.669 GB truncated to one decimal -- either way 1.6
    assert round(nbytes / 2**30, 1) == g["gbytes_even_sites"][0]
    assert int(nbytes / 1e8) / 10 == g["gbytes_even_sites"][0]


def test_compulsory_model():
    m = _model()
    assert m.compulsory_bytes_per_site("f64", 18) == 1248
    assert m.compulsory_bytes_per_site("f32", 18) == 624
    assert m.compulsory_bytes_per_site("f32", 12) == 432
    assert m.compulsory_bytes_per_site("f16", 12) == 224
    assert m.compulsory_bytes_per_site("f32", 12, extra_fields=1) == 456
    # A with fused d^dag A d: 2L + 5S per site (L = 8 links)
    assert 2 * 8 * 48 + 5 * 24 == 888
    assert m.cg_iteration_bytes_per_site("f32", 12) == 1104
    assert m.A_FLOPS_PER_SITE == 1164
