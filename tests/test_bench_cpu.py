"""Host logic of bench.py that needs no GPU: argument defaults and the lookup of
the ncu DRAM traffic from the committed profile summaries."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _parse(argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench.parse()


def test_rayleigh_default_follows_the_dimension(monkeypatch):
    assert _parse([], monkeypatch).Ra == 1e8                      # 2-D cavity workload
    assert _parse(["--dim", "3", "--n", "256"], monkeypatch).Ra == 1e7   # 3-D cavity workload
    assert _parse(["--dim", "3", "--Ra", "1e5"], monkeypatch).Ra == 1e5


@pytest.fixture
def fake_tree(tmp_path, monkeypatch):
    """A repository root with stand-in kernel sources and a profiles folder."""
    csrc = tmp_path / "paper_2509_01099_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for dim in (2, 3):
        for name in bench.KERNEL_SOURCES[dim]:
            (csrc / name).write_text(f"// {name}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _summary(root, name, sha, traffic, nodes=None):
    lines = [f"# {name}", "", f"- source_sha256: `{sha}` (sources)",
             f"- traffic_bytes_per_launch: {traffic}"]
    if nodes is not None:
        lines.append(f"- nodes_per_launch: {nodes}")
    (root / "profiles" / name).write_text("\n".join(lines) + "\n")


def test_profile_traffic_exact_size(fake_tree):
    _summary(fake_tree, "step2d_fp32_tanh1024.md", bench.kernel_source_sha(2), 69809408)
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) == 69809408
    # another size: the summary does not state its node count, so nothing is scaled
    assert bench.profile_traffic(2, "fp32", "tanh", 4096) is None
    assert bench.profile_traffic(2, "bf16dev", "tanh", 1024) is None


def test_profile_traffic_scaled_by_stated_nodes(fake_tree):
    _summary(fake_tree, "step3d_fp32_tanh128.md", bench.kernel_source_sha(3), 1000,
             nodes=128 ** 3)
    assert bench.profile_traffic(3, "fp32", "tanh", 128) == 1000
    assert bench.profile_traffic(3, "fp32", "tanh", 256) == pytest.approx(8000)


def test_profile_traffic_ignores_a_stale_source_hash(fake_tree):
    _summary(fake_tree, "step2d_fp32_tanh1024.md", "0" * 64, 123)
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) is None
    # a kernel source edited after the capture also makes the summary stale
    _summary(fake_tree, "step2d_fp32_tanh1024.md", bench.kernel_source_sha(2), 123)
    src = fake_tree / "paper_2509_01099_gb300" / "csrc" / bench.KERNEL_SOURCES[2][0]
    src.write_text(src.read_text() + "// edited\n")
    assert bench.profile_traffic(2, "fp32", "tanh", 1024) is None


def test_clock_sampler_names_the_gpu_the_rank_runs_on(monkeypatch):
    """nvidia-smi numbers physical GPUs and ignores CUDA_VISIBLE_DEVICES: the
    sampler's selector is the device's UUID, else its PCI bus id, else the
    visible-devices entry of the rank's local index."""
    import torch

    class Props:
        uuid = "1234abcd-0000-1111-2222-333344445555"
        pci_domain_id, pci_bus_id, pci_device_id = 0, 0x1B, 0

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: Props())
    assert bench.gpu_selector(0) == "GPU-1234abcd-0000-1111-2222-333344445555"
    Props.uuid = ""
    assert bench.gpu_selector(0) == "00000000:1B:00.0"

    def unavailable(i):
        raise RuntimeError("no CUDA")

    monkeypatch.setattr(torch.cuda, "get_device_properties", unavailable)
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,7")
    assert bench.gpu_selector(1) == "7"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_selector(2) == "2"


class _FakeSolver:
    """Stands in for a solver whose volume-averaged Nu relaxes as 1 + e^(-t/tau)
    in time steps, with tau set by the storage precision."""
    TAU = {"fp64": 20_000.0, "fp32": 20_000.0, "fp16neq": 20_000.0, "bf16dev": 2e12}

    def __init__(self, xi_x, xi_y, Ra, precision):
        import types
        self.t, self.prec = 0, precision
        self.info = types.SimpleNamespace(kernel=1 if precision == "fp64" else 4)

    def step(self, n):
        self.t += n

    def reduce(self, check=True):
        import math
        tau = self.TAU[self.prec]
        # BF16DEV: a slow drift that never settles to the tolerance
        nu = 1.0 + math.exp(-self.t / tau) if tau < 1e9 else 1.0 + self.t * 1e-8
        return {"Nu": nu, "Re": 2.0 * nu}

    def close(self):
        pass


def test_steady_precision_host_loop(monkeypatch, capsys):
    """The host-side Nu-window criterion of --steady-precision: windows of 100
    samples 1000 steps apart, steady when two window means agree to 2e-4; the
    budget caps an arm that never settles; deviations are taken against the
    FP64 and FP32 arms."""
    import json
    import types
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    pkg = types.SimpleNamespace(Solver=_FakeSolver, islbm_mesh_tanh=lambda n, a: None)
    args = types.SimpleNamespace(max_steps=600_000)
    bench.steady_precision(args, pkg, torch, count=2)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    arms = out["arms"]
    # exp(-t/2e4): the window means (samples 1e3 .. 1e5, 1.01e5 .. 2e5, ...)
    # are 1 + 0.198, 1 + 1.3e-3, 1 + 9e-6, 1 + 6e-8: the fourth is the first
    # within 2e-4 of the one before, so each cavity stops after 400k steps
    assert arms["fp64"]["steps_total"] == 2 * 400_000 and arms["fp64"]["all_steady"]
    assert arms["fp32"]["max_Nu_dev_from_fp64"] == 0.0
    assert arms["bf16dev"]["steps_total"] == 2 * 600_000 and not arms["bf16dev"]["all_steady"]
    assert arms["bf16dev"]["max_Nu_dev_from_fp64"] > 0
