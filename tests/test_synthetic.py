"""The seeded input generator (synthetic/) against independent statements
of its recipe: splitmix64 (Steele, Lea, Flood 2014) from its definition in
plain Python integers and the reference implementation's first outputs for
seed 1234567; the uniform and Box-Muller transforms; stream continuity
across chunked draws; the ellipse phantom's parameter ranges and support
inside the inscribed circle; the seed layout."""
import math

import numpy as np

import synthetic as S

MASK = (1 << 64) - 1


def splitmix64(seed, k):
    out, x = [], seed & MASK
    for _ in range(k):
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_reference_outputs():
    # the reference implementation's first outputs for seed 1234567
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [int(v) for v in S.SplitMix64(1234567).next_u64(5)] == want
    for seed in (0, 1, S.seed_for(1, 5), (1 << 64) - 1):
        assert [int(v) for v in S.SplitMix64(seed).next_u64(9)] == splitmix64(seed, 9)


def test_chunked_draws_continue_the_stream():
    a = S.SplitMix64(77)
    parts = np.concatenate([a.next_u64(3), a.next_u64(1), a.next_u64(6)])
    assert [int(v) for v in parts] == splitmix64(77, 10)


def test_uniform_and_normal_transforms():
    r = S.SplitMix64(9)
    u = r.uniform(1000)
    ref = [(v >> 11) * 2.0 ** -53 for v in splitmix64(9, 1000)]
    assert np.array_equal(u, np.array(ref)) and u.min() >= 0.0 and u.max() < 1.0
    # Box-Muller, cosine branch: k draws for u1 (as 1 - U), then k for u2
    k = 50
    raw = [(v >> 11) * 2.0 ** -53 for v in splitmix64(11, 2 * k)]
    want = [math.sqrt(-2.0 * math.log(1.0 - raw[i])) * math.cos(2.0 * math.pi * raw[k + i]) for i in range(k)]
    assert np.allclose(S.SplitMix64(11).normal(k), want, rtol=1e-14, atol=1e-14)
    z = S.SplitMix64(13).normal(200000)
    assert abs(z.mean()) < 4 / math.sqrt(200000) and abs(z.var() - 1.0) < 4 * math.sqrt(2 / 200000)


def test_phantom_recipe():
    rng = S.SplitMix64(S.seed_for(2, 3))
    es = S.draw_ellipses(rng, 40)
    for e in es:
        assert -0.3 <= e.cx <= 0.3 and -0.3 <= e.cy <= 0.3
        assert 0.03 <= e.a <= 0.2 and 0.03 <= e.b <= 0.2 and 0.0 <= e.phi <= math.pi and 0.0 <= e.rho < 1.0
        assert math.hypot(e.cx, e.cy) + max(e.a, e.b) <= 0.45
    n = 96
    img = S.phantom(n, 20, S.seed_for(2, 3)).reshape(n, n)
    assert np.array_equal(img, S.phantom(n, 20, S.seed_for(2, 3)).reshape(n, n))
    assert img.min() >= 0.0 and img.max() > 0.0
    c = -0.5 + (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c)
    assert not img[np.hypot(X, Y) > 0.45].any()          # inside the inscribed circle
    assert not np.array_equal(img, S.phantom(n, 20, S.seed_for(2, 4)).reshape(n, n))


def test_seed_layout_and_noise_streams():
    assert S.seed_for(3, 7) == 0x5EED0000 + 3007
    s = S.seed_for(1, 0)
    assert np.array_equal(S.noise_draws(10, s), S.SplitMix64(s + (1 << 32)).normal(10))
    u = S.uniform_noise_draws(10, s)
    assert u.min() >= -1.0 and u.max() < 1.0
