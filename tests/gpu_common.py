"""Helpers shared by the GPU parity tests: run one workload through the CUDA library
(via the C-ABI binding) and through the FP64 oracle, on identical seeded inputs."""
import numpy as np

import oracle
import synth


def torch():
    import torch as T
    return T


def dev(a):
    T = torch()
    return T.from_numpy(np.ascontiguousarray(a)).cuda()


def nmse(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2))


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def small_cfg(**kw):
    """A system whose sizes are not multiples of any tile: 40 antennas, 150 data bins
    (ragged against 32-bin tiles), 7 symbols over realisations of 3 (ragged)."""
    base = dict(name="ragged", M=40, K=3, N=256, N_d=150, Q=64, S=7, S_per_real=3,
                pa_nominal=synth.PA_NOMINAL_MP135, G=13, L_U=2, K_S=2)
    base.update(kw)
    return synth.Config(**base)


class Case:
    """Inputs on host and device, oracle ZF, and a plan."""

    def __init__(self, cfg, S=None, fc_scale=0.3, pa=None, residual=1, precision=0, max_symbols=None):
        import paper_2205_05158_gb300 as fd
        T = torch()
        self.cfg = cfg
        self.w = synth.make_workload(cfg, S=S, fc_scale=fc_scale, pa_override=pa)
        self.S = self.w.s.shape[0]
        self.R = self.w.H.shape[0]
        self.d = oracle.dims_from_config(cfg, self.w.P_T, residual)
        self.plan = fd.Plan.from_config(cfg, self.w.P_T, max_symbols=max_symbols or self.S,
                                        precision=precision, residual=residual)
        self.s = dev(self.w.s)
        self.H = dev(self.w.H)
        self.pa = dev(self.w.pa)
        self.theta = dev(self.w.theta)
        self.W = T.empty((self.R, cfg.N_d, cfg.M, cfg.K), dtype=T.complex64, device="cuda")
        self.alpha = T.empty((self.R, cfg.N_d), dtype=T.float32, device="cuda")
        self._ozf = None

    def oracle_zf(self):
        if self._ozf is None:
            self._ozf = oracle.precode(self.d, self.w.H)
        return self._ozf

    def gpu_zf(self):
        self.plan.precode(self.H, self.W, self.alpha)
        return self.W, self.alpha

    def use_oracle_zf_on_gpu(self):
        W, al = self.oracle_zf()
        self.W.copy_(dev(W.astype(np.complex64)))
        self.alpha.copy_(dev(al.astype(np.float32)))

    def gpu_distort(self):
        T = torch()
        y = T.empty_like(self.s)
        met = T.zeros(5, dtype=T.float64, device="cuda")
        self.plan.distort(self.s, self.H, self.W, self.alpha, self.pa, self.theta, y, met)
        T.cuda.synchronize()
        return y.cpu().numpy(), met.cpu().numpy()

    def gpu_backward(self):
        T = torch()
        g = T.empty(self.plan.theta_len, dtype=T.float32, device="cuda")
        met = T.zeros(5, dtype=T.float64, device="cuda")
        self.plan.backward(self.s, self.H, self.W, self.alpha, self.pa, self.theta, g, met)
        T.cuda.synchronize()
        return g.cpu().numpy(), met.cpu().numpy()

    def oracle_inputs_from_gpu_zf_free(self):
        """W / alpha the oracle uses: its own FP64 ZF."""
        return self.oracle_zf()
