"""Run bench.py's GPU arm end to end on the CPU, as a check of its host
logic (names, keys, shapes, the JSON line), not as a measurement.

torch.cuda is replaced by no-op events, streams and graphs. Tensors live on
the CPU. The library is replaced by a recorder that returns EPS_OK, writes
no outputs, and reports one contraction launch per profiled call.
Allocations are zero-filled, since nothing writes them. The cfg3 and cfg5
workloads and the cfg4 region table are shrunk to small arrays with the
same structure. bench.py is executed with its device set to the CPU, and
its one JSON line is printed as is.  Run it as a script, in its own process:
it changes torch globally."""
import contextlib
import dataclasses
import os
import sys
import types

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch  # noqa: E402

from paper_2505_03352_gb300 import epschain as eb  # noqa: E402
from paper_2505_03352_gb300 import synth  # noqa: E402

def main():
    CPU = torch.device("cpu")
    launch_count = {"n": 0, "total": 0}


    class FakeStream:
        def __init__(self, *a, **k):
            self.device = CPU
            self.cuda_stream = 0

        def wait_stream(self, s):
            pass

        def wait_event(self, e):
            pass

        def synchronize(self):
            pass


    class FakeEvent:
        def __init__(self, *a, **k):
            pass

        def record(self, *a, **k):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 0.05


    class FakeGraph:
        def replay(self):
            pass


    CUR = FakeStream()
    fake_cuda = {
        "set_device": lambda *a, **k: None,
        "synchronize": lambda *a, **k: None,
        "current_stream": lambda *a, **k: CUR,
        "Stream": FakeStream,
        "stream": lambda s: contextlib.nullcontext(),
        "Event": FakeEvent,
        "CUDAGraph": FakeGraph,
        "graph": lambda *a, **k: contextlib.nullcontext(),
        "empty_cache": lambda: None,
        "current_device": lambda: None,
    }
    for k, v in fake_cuda.items():
        setattr(torch.cuda, k, v)
    torch.Tensor.pin_memory = lambda self, *a, **k: self
    # the recorder writes no outputs: hand out zeroed memory instead of garbage
    _zeros, _zeros_like = torch.zeros, torch.zeros_like
    # (no pinned host memory without a driver: pin_memory=True is dropped)
    torch.empty = lambda *a, **k: _zeros(*a, **{n: v for n, v in k.items() if n != "pin_memory"})
    torch.empty_like = lambda *a, **k: _zeros_like(*a, **k)


    class FakeLib:
        """Every entry returns EPS_OK; eps_profile_stop reports one contraction
        launch per profiled step so the roofline arithmetic has numbers, and
        eps_launch_count four launches per call."""

        def __getattr__(self, name):
            def entry(*args):
                if name == "eps_profile_stop":
                    arr, _, n = args
                    arr[0].name = b"eps_vjp_contract"
                    arr[0].launches = max(launch_count["n"], 1)
                    arr[0].total_ms = 0.015 * max(launch_count["n"], 1)
                    n._obj.value = 1
                    launch_count["n"] = 0
                elif name == "eps_profile_start":
                    launch_count["n"] = 0
                elif name == "eps_launch_count":
                    args[0]._obj.value = launch_count["total"]
                elif name.startswith("eps_vjp") or name.startswith("eps_forward"):
                    launch_count["n"] += 1
                    launch_count["total"] += 4
                return eb.EPS_OK
            return entry


    eb._lib = FakeLib()
    eb._DEVICE_TYPE = "cpu"
    import paper_2505_03352_gb300 as ec_pkg  # noqa: E402
    _opt_init = eb.eps_opt_init
    ec_pkg.eps_opt_init = eb.eps_opt_init = lambda opt, state=None, device=None, stream=None: \
        _opt_init(opt, state, device or "cpu", stream)

    # shrink the large workloads (same code paths, small arrays)
    small = {3: dict(mx=120, my=96, nz=32), 5: dict(mx=96, my=80, nz=32)}
    for c, kw in small.items():
        synth.WORKLOADS[c] = dataclasses.replace(synth.WORKLOADS[c], **kw)
    _orig_regions = synth.batched_regions
    synth.batched_regions = lambda *a, **k: _orig_regions(n=6, lo=16, hi=64)

    # bench.py with its device mapped to the CPU
    BENCH = os.path.join(sys.path[0], "bench.py")
    src = open(BENCH).read()
    assert src.count('torch.device("cuda", local)') == 1
    src = src.replace('torch.device("cuda", local)', 'torch.device("cpu")')
    bench = types.ModuleType("bench_h")
    bench.__file__ = BENCH
    exec(compile(src, BENCH, "exec"), bench.__dict__)
    bench.L2_FLUSH_BYTES = 1 << 20

    argv = sys.argv[1:] or ["--steps", "3", "--warmup", "3", "--e2e-steps", "2"]
    sys.argv = ["bench.py"] + argv
    bench.main()


if __name__ == "__main__":
    main()
