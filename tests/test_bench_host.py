"""Host logic of bench.py that needs no GPU: the clock summary taken from the
nvidia-smi samples of the timed region (median SM clock, maximum clock, the
throttle reasons seen, malformed or unavailable samples skipped)."""
import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s


def test_clock_summary_median_max_and_reasons():
    lines = ['2070, 2070, 910.2, Not Active, Not Active, Not Active, Not Active\n',
             '2055, 2070, 1390.0, Not Active, Not Active, Not Active, Active\n',
             '1980, 2070, 1400.0, Not Active, Not Active, Not Active, Active\n']
    s = _sampler(lines).summary()
    assert s == {'sm_mhz': 2055.0, 'sm_max_mhz': 2070.0, 'reasons': ['sw_power_cap'], 'samples': 3}


def test_clock_summary_flags_thermal_and_skips_bad_samples():
    lines = ['[N/A], 2070, 900, Not Active, Not Active, Not Active, Not Active\n',
             'garbage\n',
             '1500, 2070, 800, Active, Not Active, Active, Not Active\n']
    s = _sampler(lines).summary()
    assert s['samples'] == 1 and s['sm_mhz'] == 1500.0
    assert s['reasons'] == ['hw_slowdown', 'sw_thermal_slowdown']


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s == {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': [], 'samples': 0}


def test_peak_sources_measured_and_fallback():
    got = bench.peak_sources({'hbm_gbs': 6683.2, 'sm_max_mhz': 2070.0})
    assert got == {'hbm_gbs': 6683.2, 'hbm_source': 'measured', 'sm_max_mhz': 2070.0, 'clock_source': 'measured'}
    got = bench.peak_sources({})
    assert got['hbm_gbs'] == 6800.0 and got['hbm_source'].startswith('fallback')
    assert got['sm_max_mhz'] == 2070.0 and got['clock_source'].startswith('nominal')
