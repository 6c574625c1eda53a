"""Host logic of the benchmark (no GPU): how a class's quartets are split into
launches, and the work model behind its rates."""
import pytest

import bench
from paper_2405_01834_gb300 import flops, inputs


@pytest.mark.parametrize("l", range(1, 7))
@pytest.mark.parametrize("sms", [152, 148])
def test_chunks_cover_the_class_in_whole_waves(l, sms):
    """Chunks of one class cover all 50,176 quartets; each chunk's output fits
    the buffer (up to the stated 12.5 % allowance); a class that needs several
    chunks of at least two waves gets whole waves of the SM count."""
    n = 224 * 224
    cq = bench.chunk_quartets(l, n, sms)
    per_q = inputs.ncart(l) ** 4 * 8
    assert 1 <= cq <= n
    assert cq * per_q <= bench.CHUNK_BYTES * 1.125 or cq == 1
    starts = list(range(0, n, cq))
    assert sum(min(cq, n - s) for s in starts) == n
    if n > cq and cq >= 2 * sms:
        assert cq % sms == 0


def test_model_flops_is_the_table1_model():
    for l in range(1, 7):
        assert bench.model_flops(l, 3) == 3 * flops.eri4_flops(l, l, l, l)


def test_whole_job_rate_is_weak_scaling():
    assert bench.whole_job_rate(100.0, 1, 1000.0) == pytest.approx(100.0)
    assert bench.whole_job_rate(100.0, 4, 2000.0) == pytest.approx(200.0)


@pytest.mark.parametrize("n_aux", [1, 50, 64, 600, 2300])
@pytest.mark.parametrize("n_pairs", [1, 7, 128, 4096, 100000])
@pytest.mark.parametrize("target", [8192, 65536, 262144])
def test_df_grid_fills_to_its_target(n_aux, n_pairs, target):
    """A class's density-fitting timing grid stays inside the class (distinct shells and pairs), comes within
    one column of auxiliary shells of the target triplet count (or takes the whole class when it is smaller),
    and overshoots the target by less than one row of pairs."""
    na, npr = bench.df_grid(n_aux, n_pairs, target)
    assert 1 <= na <= n_aux and 1 <= npr <= n_pairs
    assert na * npr > min(target, n_aux * n_pairs) - na or (na == n_aux and npr == n_pairs)
    assert na * npr < target + npr or na <= 64


def test_reference_arm_line(monkeypatch, capsys):
    """`bench.py --impl reference` (the oracle on the host cores, no GPU): one JSON line with the keys the
    run's contract names, the same workload config as the GPU arm, and its e2e equal to its value."""
    import json
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--classes", "1", "--steps", "1",
                                     "--warmup", "0", "--cpu-sample", "0.002"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    args = bench.parse()
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == bench.sweep_config(args, 1)
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
