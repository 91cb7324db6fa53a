"""Host-side pieces of bench.py: the algorithmic byte counts behind the
roofline figures (no GPU needed)."""
import bench


def test_complex_step_bytes_cgl_2048():
    # 2048^2 under 2/3 truncation: 1365 carried x-columns (|a_x| <= 682); SETD2 carries F_prev on them
    rows, cols = bench.algorithmic_bytes_complex(2048, 2048, 2, 1)
    assert rows == 2 * 1365 * 2048 * 8
    assert cols == (2 * 1365 + 2 * 2048 + 2 * 1365) * 2048 * 8
    # four replicas: 179 MB for the row pass, 626 MB for the column pass
    assert round(4 * rows / 1e6, 1) == 178.9 and round(4 * cols / 1e6) == 626
    # without truncation every column is carried; SETD1 has no history
    assert bench.algorithmic_bytes_complex(1024, 1024, 1, 0) == (2 * 1024 * 1024 * 8, 4 * 1024 * 1024 * 8)


def test_complex_carried_columns_match_the_mask():
    # the count of a_x in [0, nx) whose signed index satisfies 3 |a_x| < nx
    for nx in (16, 64, 1024, 2048):
        n = sum(1 for a in range(nx) if 3 * min(a, nx - a) < nx)
        rows, _ = bench.algorithmic_bytes_complex(nx, 1, 1, 1)
        assert rows == 2 * n * 8


def test_real_step_bytes_headline():
    # Model B 1024^2: 342 carried columns of the 513 stored ones; 18.7 B/site for the two passes
    w = bench.W.model_b_1024()
    rows, cols = bench.algorithmic_bytes(w, 1, 342)
    assert rows == 2 * 342 * 1024 * 8 and cols == (2 * 342 + 2 * 513) * 1024 * 8
    assert abs((rows + cols) / 1024 ** 2 - 18.703125) < 1e-12


def test_roofline_entry():
    e = bench.hbm_roofline("k", 2e9, 1.0)
    assert abs(e["achieved"] - 2000.0) < 1e-9 and abs(e["frac"] - 2000.0 / e["peak"]) < 1e-12


def test_observation_count_matches_the_timed_loop():
    # the GPU arm steps in chunks of obs_every and observes after each full chunk, at most n_obs times
    for K in (1, 5, 20, 99, 100, 101, 250, 2000, 2050):
        n_obs, obs_every = bench.observations(K)
        done = taken = 0
        while done < K:
            n = min(obs_every, K - done)
            done += n
            if n == obs_every and taken < n_obs:
                taken += 1
        assert taken == n_obs >= 1, K
        assert obs_every == min(100, K)


def test_both_arms_name_the_same_workload():
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--steps", "2", "--warmup", "0",
                          "--n", "64"], capture_output=True, text=True, timeout=300, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    w = bench.W.model_b_1024(n=[64, 64], scheme=1, h=0.05, replicas=64)
    assert line["impl"] == "reference" and line["config"] == bench.headline_config(w, 64, 1, 2)
    assert line["steps"] == 2 and line["warmup"] == 0 and line["e2e"]["h2d_bytes_per_step"] == 0
