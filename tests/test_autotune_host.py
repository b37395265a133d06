"""Host logic of the autotuner's pool sizing: tickets are pixels x the bins
that receive samples, candidate pools are clamped powers of two near a
fraction of the tickets, and a fraction found on a reduced-sample probe is
applied to the full views' tickets."""
from paper_2303_15762_gb300 import autotune


def _v(side, spp, bins):
    return dict(width=side, height=side, spp=spp, n_bins=bins)


def test_tickets_count_bins_with_samples():
    assert autotune.tickets([_v(4, 16, 32)]) == 16 * 16  # spp < bins: one ticket per sample
    assert autotune.tickets([_v(4, 256, 32)]) == 16 * 32  # every bin has samples
    assert autotune.tickets([_v(2, 3, 8), _v(3, 8, 4)]) == 4 * 3 + 9 * 4


def test_pool_for_is_a_clamped_power_of_two():
    for n in (1, 10_000, 3_000_000, 303_000_000, 10 ** 12):
        for f in autotune.POOL_FRACTIONS:
            p = autotune.pool_for(f, n)
            assert p & (p - 1) == 0
            assert autotune.POOL_MIN <= p <= autotune.POOL_MAX
    assert autotune.pool_for(1 / 8, 1 << 28) == 1 << 25
    assert autotune.pool_for(1 / 8, 100) == autotune.POOL_MIN
    assert autotune.pool_for(1.0, 10 ** 12) == autotune.POOL_MAX


def test_probe_fraction_scales_to_the_full_views():
    full = [_v(1024, 16, 32)] * 4
    probe = [dict(v, spp=4) for v in full]
    n_full, n_probe = autotune.tickets(full), autotune.tickets(probe)
    assert n_full == 4 * n_probe
    p_probe = autotune.pool_for(1 / 16, n_probe)
    assert autotune.pool_for(p_probe / n_probe, n_full) == 4 * p_probe
