"""Several supercell partitions in one plan (the batched layout of Sec. IV: independent
partitions of uneven size), checked element by element against the FP64 oracle.

  grouped  the last flush of every stream goes out as one tensor-core launch over all
           streams (tiles ordered longest first); parity per stream and the launch count
  graph    reset + pushes + finalize_async of a whole segment captured into a CUDA graph;
           two replays over two different frame sets, each against the oracle
  tune     tiles picked by the autotuner (timed candidates, then a cache file hit), parity
"""
import numpy as np
import pytest

import oracle
from synth import Detector, StreamSpec
from tests.helpers import oracle_kw, rel_err_peak, stream_config

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-5}

# uneven probes, ROIs (one rectangular), segment lengths (ragged against every block size),
# energy grids and windows
SPECS = [
    StreamSpec(P=3, Kx=48, Ky=48, T=200, Tc=40, n_omega=70, E_max_meV=120.0, window="hann",
               detectors=(Detector(r_out=10.0),)),
    StreamSpec(P=2, Kx=40, Ky=24, T=96, Tc=32, fft_bins=48, window="gauss",
               detectors=(Detector(r_out=6.0), Detector("annular", 2.0, -1.0, 3.0, 9.0))),
    StreamSpec(P=5, Kx=32, Ky=32, T=333, Tc=50, n_omega=120, E_max_meV=150.0, window="rect",
               detectors=()),
    StreamSpec(P=1, Kx=64, Ky=64, T=64, Tc=64, n_omega=9, E_max_meV=90.0, window="tukey",
               window_param=0.3, subtract_mean=False, bose_T_K=300.0),
]

MODES = {"split_bf16": dict(precision="split_bf16"),
         "split_inplace": dict(precision="split_bf16", frames_in_place=True),
         "fp32": dict(precision="fp32")}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02236_gb300 import build
    build.build_all()


def make_frames(spec, seed):
    rng = np.random.default_rng(seed)
    P, T, K, L = spec.P, spec.T, spec.Ky, spec.Kx
    e = rng.standard_normal((P, 1, K, L)) + 1j * rng.standard_normal((P, 1, K, L))
    s = 1e-2 * (rng.standard_normal((P, T, K, L)) + 1j * rng.standard_normal((P, T, K, L)))
    return (e + s).astype(np.complex64)


def device_frames(fr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(fr.transpose(1, 0, 2, 3))).to("cuda")  # [T][P][Ky][Kx]


def push_all(plan, bufs, stream=None):
    """Round-robin pushes of Tc frames, as partitions arrive interleaved."""
    pushed = [0] * len(SPECS)
    while any(pushed[i] < s.T for i, s in enumerate(SPECS)):
        for i, s in enumerate(SPECS):
            if pushed[i] < s.T:
                n = min(s.Tc, s.T - pushed[i])
                fb = s.P * s.Kx * s.Ky * 8
                plan.push(i, bufs[i].data_ptr() + pushed[i] * fb, n, cuda_stream=stream)
                pushed[i] += n


def check_all(plan, I, S, frames, tol):
    worst = 0.0
    for i, s in enumerate(SPECS):
        ref = oracle.forward(frames[i], **oracle_kw(s))
        io, so = plan.offsets(i)
        n = s.P * s.Nw * s.Ky * s.Kx
        got = I[io:io + n].cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx)
        e = rel_err_peak(got, ref.I)
        assert e <= tol, (i, e)
        worst = max(worst, e)
        D = len(s.detectors)
        if D:
            gs = S[so:so + s.P * D * s.Nw].cpu().numpy().reshape(s.P, D, s.Nw)
            es = rel_err_peak(gs, ref.S)
            assert es <= tol, (i, es)
    return worst


@pytest.mark.parametrize("mode", sorted(MODES))
def test_grouped_final_flush(mode):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    kw = MODES[mode]
    frames = [make_frames(s, 100 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    with TacawPlan([stream_config(s) for s in SPECS], **kw) as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        push_all(plan, bufs)
        before = plan.info()["kernel_launches"]
        plan.finalize(I, S)
        after = plan.info()
        worst = check_all(plan, I, S, frames, TOL[kw["precision"]])
    n_det = sum(1 for s in SPECS if len(s.detectors))
    if mode == "split_bf16":
        bf = after["tc_block_frames"]
        tails = sum(1 for s in SPECS if s.T % bf)
        # mean residual per stream, zero tails, ONE contraction launch, one aperture launch per stream
        assert after["kernel_launches"] - before == len(SPECS) + tails + 1 + n_det
    assert after["flushes"] == len(SPECS)
    print(f"{mode}: worst max rel I error {worst:.3g}")


@pytest.mark.parametrize("mode", ["split_bf16", "split_inplace", "fp32"])
def test_graph_capture_and_replay(mode):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    kw = MODES[mode]
    tol = TOL[kw["precision"]]
    frames = [make_frames(s, 200 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    st = torch.cuda.Stream()
    with TacawPlan([stream_config(s) for s in SPECS], **kw) as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        # one eager segment on the capture stream first (kernel attributes set outside capture)
        with torch.cuda.stream(st):
            plan.reset(st)
            push_all(plan, bufs, st)
            plan.finalize_async(I, S, cuda_stream=st)
            plan.check_errors(st)
        check_all(plan, I, S, frames, tol)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            cur = torch.cuda.current_stream()
            plan.reset(cur)
            push_all(plan, bufs, cur)
            plan.finalize_async(I, S, cuda_stream=cur)
        launches = plan.info()["kernel_launches"]
        for rep, seed in enumerate((300, 400)):
            frames = [make_frames(s, seed + i) for i, s in enumerate(SPECS)]
            for b, f in zip(bufs, frames):
                b.copy_(device_frames(f))
            I.zero_()
            S.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            plan.check_errors(torch.cuda.current_stream())
            worst = check_all(plan, I, S, frames, tol)
            print(f"{mode} replay {rep}: worst max rel I error {worst:.3g}")
        # replays launch from the graph, not through the library
        assert plan.info()["kernel_launches"] == launches
        del g


@pytest.mark.parametrize("kw", [dict(precision="split_bf16", tc_max_ctas=7),
                                dict(precision="split_bf16", tc_max_ctas=3, frames_in_place=True)])
def test_capped_persistent_grid(kw):
    """Persistent contraction grids capped at a few CTAs (each walks many tiles of several
    streams; the capped last flush runs on the plan's forked high-priority stream)."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frames = [make_frames(s, 700 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    st = torch.cuda.Stream()
    with TacawPlan([stream_config(s) for s in SPECS], **kw) as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        with torch.cuda.stream(st):
            push_all(plan, bufs, st)
            plan.finalize(I, S, cuda_stream=st)
        torch.cuda.synchronize()
        worst = check_all(plan, I, S, frames, TOL["split_bf16"])
    print(f"capped grid {kw}: worst max rel I error {worst:.3g}")


def test_autotuned_tiles_and_cache(tmp_path):
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frames = [make_frames(s, 500 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    cache = str(tmp_path / "tiles.txt")
    infos = []
    for rep in range(2):
        with TacawPlan([stream_config(s) for s in SPECS], precision="split_bf16", tune=cache) as plan:
            info = plan.info()
            infos.append(info)
            I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
            S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
            push_all(plan, bufs)
            plan.finalize(I, S)
            worst = check_all(plan, I, S, frames, TOL["split_bf16"])
        print(f"tuned plan {rep}: {info['tune_candidates']} candidates timed in {info['tune_ms']:.1f} ms, "
              f"worst error {worst:.3g}")
        assert info["tuned_streams"] == len(SPECS)
    assert infos[0]["tune_candidates"] > 0
    assert infos[1]["tune_candidates"] == 0            # every shape came from the cache
    assert infos[1]["omega_tile"] == infos[0]["omega_tile"]
    lines = open(cache).read().splitlines()
    assert len(lines) == len(SPECS)
    for ln in lines:                                   # "<shape key> | <wt>:<ms> ..."
        key, table = ln.split(" | ")
        cands = [tuple(map(float, c.split(":"))) for c in table.split()]
        assert key.startswith("tacaw-tune-v2") and cands and all(c[0] % 8 == 0 and c[1] > 0 for c in cands)
    # a fixed energy tile is honoured
    with TacawPlan([stream_config(s) for s in SPECS], precision="split_bf16", tune="", tc_omega_tile=48) as plan:
        info = plan.info()
    assert info["omega_tile"] == 48 and info["tuned_streams"] == len(SPECS)


ROUNDS = [StreamSpec(P=2, Kx=24, Ky=24, T=160, Tc=32, n_omega=50, E_max_meV=120.0, window="hann",
                     detectors=(Detector(r_out=6.0),)),
          StreamSpec(P=3, Kx=16, Ky=20, T=96, Tc=32, n_omega=30, E_max_meV=90.0, window="gauss",
                     detectors=(Detector(r_out=4.0),)),
          StreamSpec(P=1, Kx=32, Ky=32, T=224, Tc=32, n_omega=70, E_max_meV=150.0, window="hann",
                     detectors=())]


@pytest.mark.parametrize("capture", [False, True], ids=["eager", "graph"])
def test_flush_rounds_share_launches(capture):
    """K_stage = 64 < T: the partitions' rings fill in the same push round (32 frames per stream
    per round).  Each round's flushes go out as one grouped launch at the next push: rounds 2, 4
    and 6 fill {A, B, C}, {A, C} and {C}, then the final flushes of all three share one launch --
    4 contraction launches for 9 flushes -- and the result matches the oracle (eager and inside a
    captured CUDA graph)."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frames = [make_frames(s, 700 + i) for i, s in enumerate(ROUNDS)]
    bufs = [device_frames(f) for f in frames]
    st = torch.cuda.Stream()

    def push_rounds(plan, stream):
        pushed = [0] * len(ROUNDS)
        while any(pushed[i] < s.T for i, s in enumerate(ROUNDS)):
            for i, s in enumerate(ROUNDS):
                if pushed[i] < s.T:
                    fb = s.P * s.Kx * s.Ky * 8
                    plan.push(i, bufs[i].data_ptr() + pushed[i] * fb, s.Tc, cuda_stream=stream)
                    pushed[i] += s.Tc

    with TacawPlan([stream_config(s) for s in ROUNDS], precision="split_bf16", k_stage=64, accum="kahan") as plan:
        info = plan.info()
        assert info["k_stage"] == 64
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        f0, n0 = info["flush_launches"], info["flushes"]
        with torch.cuda.stream(st):
            plan.reset(st)
            push_rounds(plan, st)
            plan.finalize_async(I, S, cuda_stream=st)
            plan.check_errors(st)
        after = plan.info()
        assert after["flushes"] - n0 == 9
        assert after["flush_launches"] - f0 == 4
        if capture:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                cur = torch.cuda.current_stream()
                plan.reset(cur)
                push_rounds(plan, cur)
                plan.finalize_async(I, S, cuda_stream=cur)
            frames = [make_frames(s, 800 + i) for i, s in enumerate(ROUNDS)]
            for b, f in zip(bufs, frames):
                b.copy_(device_frames(f))
            I.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            plan.check_errors(torch.cuda.current_stream())
            del g
        torch.cuda.synchronize()
        worst = 0.0
        for i, s in enumerate(ROUNDS):
            ref = oracle.forward(frames[i], **oracle_kw(s))
            io, so = plan.offsets(i)
            n = s.P * s.Nw * s.Ky * s.Kx
            e = rel_err_peak(I[io:io + n].cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx), ref.I)
            assert e <= TOL["split_bf16"], (i, e)
            worst = max(worst, e)
    print(f"flush rounds ({'graph' if capture else 'eager'}): worst max rel I error {worst:.3g}")


def push_group_rounds(plan, specs, bufs, stream=None):
    """Round-robin as push_all, but each round is one tacaw_push_frames_group call."""
    pushed = [0] * len(specs)
    calls = 0
    while any(pushed[i] < s.T for i, s in enumerate(specs)):
        ids, ptrs, cnt = [], [], []
        for i, s in enumerate(specs):
            if pushed[i] < s.T:
                n = min(s.Tc, s.T - pushed[i])
                fb = s.P * s.Kx * s.Ky * 8
                ids.append(i)
                ptrs.append(bufs[i].data_ptr() + pushed[i] * fb)
                cnt.append(n)
                pushed[i] += n
        plan.push_group(ids, ptrs, cnt, cuda_stream=stream)
        calls += 1
    return calls


def test_push_group_matches_single_pushes():
    """tacaw_push_frames_group gives the same I and S, bit for bit, as one tacaw_push_frames per
    stream (the same conversion of every row, the same flushes), with fewer launches: the
    streams whose pushes are multiples of 4 frames share one conversion launch per round, the
    ragged one (50-frame pushes) goes through the single-push path.  Both match the oracle."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frames = [make_frames(s, 900 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    out = []
    for grouped in (False, True):
        with TacawPlan([stream_config(s) for s in SPECS], precision="split_bf16") as plan:
            info = plan.info()
            I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
            S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
            l0 = plan.info()["kernel_launches"]
            if grouped:
                push_group_rounds(plan, SPECS, bufs)
            else:
                push_all(plan, bufs)
            pushes = plan.info()["kernel_launches"] - l0
            plan.finalize(I, S)
            check_all(plan, I, S, frames, TOL["split_bf16"])
            out.append((I.cpu().numpy(), S.cpu().numpy(), pushes))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[1][2] < out[0][2], (out[0][2], out[1][2])


@pytest.mark.parametrize("capture", [False, True], ids=["eager", "graph"])
def test_push_group_flush_rounds(capture):
    """The flush-round workload (K_stage = 64) pushed one group per round: rings that fill in
    the same round flush together at the next group push -- 4 contraction launches for 9
    flushes, as with single pushes -- eager and inside a captured CUDA graph, against the
    oracle."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    frames = [make_frames(s, 950 + i) for i, s in enumerate(ROUNDS)]
    bufs = [device_frames(f) for f in frames]
    st = torch.cuda.Stream()
    with TacawPlan([stream_config(s) for s in ROUNDS], precision="split_bf16", k_stage=64, accum="kahan") as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        f0, n0 = info["flush_launches"], info["flushes"]
        with torch.cuda.stream(st):
            plan.reset(st)
            push_group_rounds(plan, ROUNDS, bufs, st)
            plan.finalize_async(I, S, cuda_stream=st)
            plan.check_errors(st)
        after = plan.info()
        assert after["flushes"] - n0 == 9
        assert after["flush_launches"] - f0 == 4
        if capture:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                cur = torch.cuda.current_stream()
                plan.reset(cur)
                push_group_rounds(plan, ROUNDS, bufs, cur)
                plan.finalize_async(I, S, cuda_stream=cur)
            frames = [make_frames(s, 980 + i) for i, s in enumerate(ROUNDS)]
            for b, f in zip(bufs, frames):
                b.copy_(device_frames(f))
            I.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            plan.check_errors(torch.cuda.current_stream())
            del g
        torch.cuda.synchronize()
        for i, s in enumerate(ROUNDS):
            ref = oracle.forward(frames[i], **oracle_kw(s))
            io, so = plan.offsets(i)
            n = s.P * s.Nw * s.Ky * s.Kx
            e = rel_err_peak(I[io:io + n].cpu().numpy().reshape(s.P, s.Nw, s.Ky, s.Kx), ref.I)
            assert e <= TOL["split_bf16"], (i, e)


def test_push_group_refusals_leave_the_plan_unchanged():
    """A repeated stream id, an entry past its segment's end, or an unreadable address refuses
    the whole group before any work; the plan then takes the full segment as usual."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    from paper_2607_02236_gb300.tacaw import TacawError, ERR_INVALID_ARG, ERR_OVERFLOW
    frames = [make_frames(s, 990 + i) for i, s in enumerate(SPECS)]
    bufs = [device_frames(f) for f in frames]
    with TacawPlan([stream_config(s) for s in SPECS], precision="split_bf16") as plan:
        info = plan.info()
        I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
        S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
        l0 = plan.info()["kernel_launches"]
        with pytest.raises(TacawError) as ei:
            plan.push_group([0, 0], [bufs[0], bufs[0]], [8, 8])
        assert ei.value.status == ERR_INVALID_ARG and "twice" in str(ei.value)
        with pytest.raises(TacawError) as ei:
            plan.push_group([0, 1], [bufs[0], bufs[1]], [8, SPECS[1].T + 4])
        assert ei.value.status == ERR_OVERFLOW
        host = np.zeros(64, dtype=np.complex64)
        with pytest.raises(TacawError) as ei:
            plan.push_group([0, 1], [bufs[0], host.ctypes.data], [8, 8])
        assert ei.value.status == ERR_INVALID_ARG and "d_frames" in str(ei.value)
        assert plan.info()["kernel_launches"] == l0
        push_group_rounds(plan, SPECS, bufs)
        plan.finalize(I, S)
        check_all(plan, I, S, frames, TOL["split_bf16"])


def _welch_mixed_configs():
    """SPECS with the second stream averaged over Welch segments (N = 3, stride T/2, 8 leading
    frames skipped): its pushes take the single-push path inside a group."""
    cfgs = [stream_config(s) for s in SPECS]
    s1 = SPECS[1]
    cfgs[1].welch_segments, cfgs[1].welch_stride, cfgs[1].skip_init = 3, s1.T // 2, 8
    total = [s.T for s in SPECS]
    total[1] = 8 + s1.T + 2 * (s1.T // 2)
    return cfgs, total


@pytest.mark.parametrize("mode", ["split_fp16", "fp32", "split_inplace", "welch_mixed"])
def test_push_group_every_path(mode):
    """A group push gives the same I and S, bit for bit, as single pushes on every path it can
    meet: split-FP16 (grouped conversion of scaled fp16 pieces), the FP32 path and the in-place
    path (single pushes inside the group), and a Welch stream with skipped leading frames beside
    plain streams."""
    import torch
    from paper_2607_02236_gb300 import TacawPlan
    kw = {"split_fp16": dict(precision="split_fp16"), "fp32": dict(precision="fp32"),
          "split_inplace": dict(precision="split_bf16", frames_in_place=True),
          "welch_mixed": dict(precision="split_bf16")}[mode]
    if mode == "welch_mixed":
        cfgs, total = _welch_mixed_configs()
    else:
        cfgs, total = [stream_config(s) for s in SPECS], [s.T for s in SPECS]
    rng = np.random.default_rng(1200)
    frames = []
    for s, n in zip(SPECS, total):
        e = rng.standard_normal((s.P, 1, s.Ky, s.Kx)) + 1j * rng.standard_normal((s.P, 1, s.Ky, s.Kx))
        f = e + 1e-2 * (rng.standard_normal((s.P, n, s.Ky, s.Kx)) + 1j * rng.standard_normal((s.P, n, s.Ky, s.Kx)))
        frames.append(f.astype(np.complex64))
    bufs = [device_frames(f) for f in frames]
    out = []
    for grouped in (False, True):
        with TacawPlan(cfgs, **kw) as plan:
            info = plan.info()
            I = torch.zeros(info["I_elems"], dtype=torch.float32, device="cuda")
            S = torch.zeros(max(1, info["S_elems"]), dtype=torch.float32, device="cuda")
            pushed = [0] * len(SPECS)
            while any(pushed[i] < total[i] for i in range(len(SPECS))):
                ids, ptrs, cnt = [], [], []
                for i, s in enumerate(SPECS):
                    if pushed[i] < total[i]:
                        n = min(s.Tc, total[i] - pushed[i])
                        ids.append(i)
                        ptrs.append(bufs[i].data_ptr() + pushed[i] * s.P * s.Kx * s.Ky * 8)
                        cnt.append(n)
                        pushed[i] += n
                if grouped:
                    plan.push_group(ids, ptrs, cnt)
                else:
                    for i, ptr, n in zip(ids, ptrs, cnt):
                        plan.push(i, ptr, n)
            plan.finalize(I, S)
            out.append((I.cpu().numpy(), S.cpu().numpy()))
            if mode != "welch_mixed" and grouped:
                # the plain streams against the oracle as well
                check_all(plan, I, S, frames, TOL[kw["precision"]] if kw["precision"] in TOL else 1e-5)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
