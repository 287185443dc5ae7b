"""The stylized-fact statistics of the composition sweep on traces whose
answers are known in closed form."""
import numpy as np

from paper_2606_21784_gb300 import dynamics


def _trace(prices, volume=10):
    p = np.asarray(prices, np.int32)
    t = np.zeros((1 if p.ndim == 1 else p.shape[0], p.shape[-1], 2), np.int32)
    t[:, :, 0] = p
    t[:, :, 1] = np.where(p >= 0, volume, 0)
    return t


def test_constant_price_has_no_volatility():
    f = dynamics.facts(_trace([64] * 50), L=128)
    assert f["volatility"] == 0 and f["volume_per_step"] == 10 and f["mean_price"] == 64
    assert f["price_std"] == 0


def test_steady_trend_has_no_return_volatility_but_a_price_excursion():
    f = dynamics.facts(_trace(np.arange(62, -138, -2)), L=128, window=True)  # -2 every step from 64
    assert f["volatility"] == 0
    assert abs(f["price_std"] - np.arange(62, -138, -2).std()) < 1e-12


def test_bid_ask_bounce_has_lag1_autocorrelation_minus_one():
    f = dynamics.facts(_trace([65, 64] * 200), L=128)  # returns +1, -1, +1, ...
    assert abs(f["acf_r"][0] + 1) < 0.01 and abs(f["acf_r"][1] - 1) < 0.01
    assert abs(f["volatility"] - 1) < 0.01


def test_symmetric_steps_have_excess_kurtosis_minus_two():
    rng = np.random.default_rng(0)
    steps = rng.choice([-1, 1], size=(20, 2000))
    prices = 5000 + np.cumsum(steps, axis=1)  # stays on the grid: no step reads as a missing trade
    f = dynamics.facts(_trace(prices), L=10000)
    assert abs(f["excess_kurtosis"] + 2) < 0.05  # a +/-1 coin has kurtosis 1
    assert abs(f["acf_r"][0]) < 0.02 and abs(f["acf_abs_r"][0]) < 0.02


def test_steps_without_trade_keep_the_last_price():
    f = dynamics.facts(_trace([66, -1, -1, 66, 70]), L=128)  # returns 2, 0, 0, 0, 4 from L/2 = 64
    assert f["volume_per_step"] == 6.0  # 10 on three trading steps out of five
    assert abs(f["mean_price"] - (66 + 66 + 66 + 66 + 70) / 5) < 1e-12


def test_window_traces_take_the_absolute_price_as_is():
    # a window trace records the absolute last price after every step, which
    # may be negative or far outside [0, L); returns from L/2 = 64
    t = np.zeros((1, 4, 2), np.int32)
    t[0, :, 0] = [60, -5, -5, 300]
    t[0, :, 1] = [3, 4, 0, 8]
    f = dynamics.facts(t, L=128, window=True)
    r = np.array([-4, -65, 0, 305], np.float64)
    assert abs(f["volatility"] - r.std()) < 1e-12
    assert f["volume_per_step"] == 3.75 and abs(f["mean_price"] - (60 - 5 - 5 + 300) / 4) < 1e-12


def test_oracle_sweep_momentum_runs_away_on_a_window():
    """The composition sweep's finding on the oracle itself (CPU, small): on a
    sliding window the spread of the price level grows with the momentum
    share, while without momentum the price stays near its start and returns
    reverse at lag 1 (bid-ask bounce)."""
    import oracle as o
    from paper_2606_21784_gb300 import workloads as wl

    def run(mom):
        w = wl.workload("paper_8192_256", M=6, L=128, A=128, mom_pct=mom, maker_pct=15, window=1)
        tr = np.zeros((6, 300, 2), np.int32)
        for m in range(6):
            bk = o.paper_init(m, 128, 128)
            tp, tv = o.paper_run(w["params"], bk, 0, 300)
            tr[m, :, 0], tr[m, :, 1] = tp, tv
        return dynamics.facts(tr, 128, window=True)

    f0, f50 = run(0), run(50)
    assert f50["price_std"] > 5 * f0["price_std"]
    assert f0["acf_r"][0] < -0.1 and f0["volume_per_step"] > 0
