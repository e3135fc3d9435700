"""The seeded input generator (no GPU): the SplitMix64 stream against its
published reference outputs, its counter-based splitting, the Box-Muller
normals, and the workload scenes against the sizes they stand for.  Both the
oracle and the CUDA path draw their inputs from this module, so a slip here
would go unnoticed by the parity tests."""
import numpy as np

from paper_2202_09703_gb300 import synth as S


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 (Steele, Lea and Flood 2014) for two seeds, as published with the generator
    assert [int(v) for v in S.SplitMix64(0).next_u64(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in S.SplitMix64(1234567).next_u64(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_stream_splits_without_changing_the_draws():
    a = S.SplitMix64(99)
    whole = a.next_u64(10)
    b = S.SplitMix64(99)
    parts = np.concatenate([b.next_u64(3), b.next_u64(7)])
    assert np.array_equal(whole, parts)


def test_uniform_and_normal_draws():
    u = S.SplitMix64(5).uniform(200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    z = S.SplitMix64(6).normal(200_001)
    assert z.size == 200_001 and np.all(np.isfinite(z))
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 2e-2
    k = S.SplitMix64(7).integers(3, 9, 50_000)
    assert k.min() == 3 and k.max() == 9


def test_workload_scenes_have_the_stated_sizes():
    s0, s1, s2 = S.cfg0(), S.cfg1(), S.cfg2()
    assert (s0.img_w, s0.img_h, s0.K, s0.M, len(s0.layers)) == (64, 64, 16 * 8, 512, 2)
    assert (s1.img_w, s1.img_h, s1.K, s1.M, len(s1.layers)) == (256, 512, 64 * 16, 2048, 4)
    assert (s2.img_w, s2.img_h, s2.K, s2.M, len(s2.layers)) == (512, 1024, 128 * 32, 4096, 4)
    assert abs(s1.pitch - 0.5e-3) < 1e-12 and abs(s2.pitch - 0.25e-3) < 1e-12
    assert s0.n_iter == 20 and s1.n_iter == 50 and s2.n_iter == 50
    assert [round(L.speed) for L in s1.layers] == [1480, 5900, 3000, 4500]
