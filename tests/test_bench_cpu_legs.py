"""CPU: the benchmark's CPU-baseline legs run and report what they timed.

The one-thread leg runs the oracle in a child process limited to one BLAS
thread; the spatial-route leg times the per-block IDCT + spatial filter + DCT
that the DCT-domain operator replaces.  Both are reported baselines, so the
checks are that they run, finish in bounded time and describe their sample.
"""
import bench
import datagen


def test_one_thread_and_spatial_legs():
    job = datagen.headline_job(256, 256)
    x = bench.oracle_coefficients(job)
    one = bench.cpu_oracle_one_thread(job, x, 512, 0.2)
    assert "error" not in one, one
    assert one["value"] > 0 and one["cores"] == 1 and "512 blocks" in one["sample"]
    sp = bench.cpu_spatial_route(job, 256, 0.2)
    assert sp["value"] > 0 and "256 blocks" in sp["sample"]
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
