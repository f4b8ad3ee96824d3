"""ctypes binding of libpmf.so (the C ABI declared in include/pmf.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Function names are those of the C ABI.  Importing this module
loads libpmf.so and raises if it has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmf.so")

PMF_OK, PMF_EINVAL, PMF_ENOMEM, PMF_ECUDA, PMF_ENUMERIC, PMF_ETIMEOUT, PMF_ESTATE = range(7)
STATUS_NAMES = {0: "PMF_OK", 1: "PMF_EINVAL", 2: "PMF_ENOMEM", 3: "PMF_ECUDA", 4: "PMF_ENUMERIC",
                5: "PMF_ETIMEOUT", 6: "PMF_ESTATE"}
PMF_MODEL_1D_DOUBLEWELL, PMF_MODEL_CHAIN = 0, 1
PMF_FP32, PMF_FP64 = 0, 1
PMF_WORK_PER_WINDOW_INCREMENT, PMF_WORK_PAIRED_CUMULATIVE = 0, 1
PMF_BATCH_GRAPH, PMF_BATCH_PACKED = 0, 1

_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I64 = C.POINTER(C.c_int64)


class PmfError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SystemDesc(C.Structure):
    _fields_ = [("model", C.c_int), ("precision", C.c_int), ("n_chains", C.c_int),
                ("n_beads", C.POINTER(C.c_int)), ("sigma", _D), ("epsilon", _D), ("charge", _D),
                ("mass", _D), ("dih_k", _D), ("dih_phase", _D), ("pos0", _D),
                ("bond_k", C.c_double), ("bond_r0", C.c_double), ("angle_k", C.c_double),
                ("angle_theta0", C.c_double), ("coulomb_k", C.c_double), ("nonbonded", C.c_int),
                ("dw_a", C.c_double), ("x0", C.c_double)]


class RunParams(C.Structure):
    _fields_ = [("k", C.c_double), ("kT", C.c_double), ("dt", C.c_double), ("gamma", C.c_double),
                ("n_steps", C.c_int64), ("n_steps_per_window", _I64), ("n_equil", C.c_int64),
                ("sample_stride", C.c_int), ("replicas", C.c_int), ("seed", C.c_uint64),
                ("uid_base", C.c_uint32), ("chain", C.c_int), ("timeout_s", C.c_double),
                ("segment_wait_s", C.c_double)]


MAX_RUN_WINDOWS = 4096  # PMF_MAX_RUN_WINDOWS


class BatchItem(C.Structure):
    _fields_ = [("chain", C.c_int), ("n_windows", C.c_int), ("lambda_", _D)]


class HistParams(C.Structure):
    _fields_ = [("x_lo", C.c_double), ("dx", C.c_double), ("n_x", C.c_int), ("dw", C.c_double), ("M", C.c_int),
                ("left_edge", C.c_int)]


class RunInfo(C.Structure):
    _fields_ = [("n_windows", C.c_int), ("replicas", C.c_int), ("total_samples", C.c_int64),
                ("samples_per_window", C.c_int64 * MAX_RUN_WINDOWS),
                ("sample_offset", C.c_int64 * MAX_RUN_WINDOWS)]


RESULT_FIELDS = ("lambda", "dF_JE", "dF_fluct", "dF_G", "dF_com", "uncertainty", "se_JE",
                 "se_fluct", "var_ZW", "W_mean", "acc_force", "mean_x", "var_x", "gamma2")


class FreeEnergyResult(C.Structure):
    _fields_ = [("capacity", C.c_int)] + [(("lambda_" if f == "lambda" else f), _D) for f in RESULT_FIELDS]


_IP = C.POINTER(C.c_int)


class AdaptiveTrace(C.Structure):
    _fields_ = [("max_rounds", C.c_int), ("max_windows", C.c_int), ("replicas", C.c_int), ("rounds", C.c_int),
                ("n_windows", _IP), ("n_inserted", _IP), ("lambda_", _D), ("mu", _D), ("log_var", _D),
                ("ovl", _D), ("inserted", _D), ("target", _D), ("cand_x", _D), ("seed", _IP),
                ("data_ovl", _D), ("trained", _IP)]


class AdaptiveParams(C.Structure):
    _fields_ = [("overlap_threshold", C.c_double), ("max_rounds", C.c_int), ("max_windows", C.c_int),
                ("mlp_steps", C.c_int), ("mlp_batch", C.c_int), ("mlp_lr", C.c_double), ("mlp_seed", C.c_uint64),
                ("mlp_init", _F), ("trace", C.POINTER(AdaptiveTrace)), ("continue_windows", C.c_int),
                ("train_on_gap", C.c_int)]


class AdaptiveInfo(C.Structure):
    _fields_ = [("n_windows", C.c_int), ("rounds", C.c_int), ("inserted", C.c_int), ("gpu_seconds", C.c_double),
                ("mlp_loss", C.c_double), ("lambda_", C.c_double * 1024)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1105_4840_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.pmf_create_system.argtypes = [C.POINTER(SystemDesc), C.POINTER(P)]
    L.pmf_destroy_system.argtypes = [P]
    L.pmf_destroy_system.restype = None
    for name in ("pmf_run_windows", "pmf_run_prepare"):
        getattr(L, name).argtypes = [P, _D, C.c_int, C.POINTER(RunParams), C.POINTER(P)]
    L.pmf_run_prepare_seeded.argtypes = [P, _D, C.c_int, C.POINTER(RunParams), _D, C.POINTER(P)]
    L.pmf_run_prepare_sequential.argtypes = [P, _D, C.c_int, C.POINTER(RunParams), C.POINTER(P)]
    L.pmf_run_prepare_smd.argtypes = [P, C.c_double, C.c_double, C.POINTER(RunParams), C.POINTER(P)]
    L.pmf_smd_work.argtypes = [P, _D, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pmf_smd_free_energy.argtypes = [P, _D, _D, _D, _D, _D, _D, C.c_int]
    L.pmf_run_batch_prepare.argtypes = [P, C.POINTER(BatchItem), C.c_int, C.POINTER(RunParams), C.POINTER(P)]
    L.pmf_free_energy_item.argtypes = [P, C.c_int, C.POINTER(FreeEnergyResult)]
    L.pmf_run_launch.argtypes = [P]
    L.pmf_run_wait.argtypes = [P]
    L.pmf_destroy_run.argtypes = [P]
    L.pmf_destroy_run.restype = None
    L.pmf_get_run_info.argtypes = [P, C.POINTER(RunInfo)]
    L.pmf_x_samples.argtypes = [P, _F, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pmf_work_samples.argtypes = [P, C.c_int, _D, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pmf_free_energy.argtypes = [P, C.POINTER(FreeEnergyResult)]
    L.pmf_free_energy_from_samples.argtypes = [C.c_void_p, C.c_int, _D, C.c_int, C.c_int, _I64,
                                               C.c_double, C.c_double, C.POINTER(FreeEnergyResult)]
    L.pmf_work_distributions.argtypes = [P, C.POINTER(HistParams), _D, C.c_size_t, _D, _D, _D]
    L.pmf_run_partials.argtypes = [P, _D, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pmf_free_energy_from_partials.argtypes = [_D, _D, C.c_int, C.c_int, C.c_double, C.c_double,
                                                C.POINTER(FreeEnergyResult)]
    L.pmf_final_state.argtypes = [P, _D, _D, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pmf_philox.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int,
                             C.POINTER(C.c_uint32), _F]
    L.pmf_chain_forces.argtypes = [P, C.c_int, _D, C.c_double, C.c_double, _D]
    L.pmf_chain_schedule.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_size_t,
                                     C.POINTER(C.c_size_t), C.POINTER(C.c_int)]
    L.pmf_run_reduce.argtypes = [P]
    L.pmf_run_set_queue_start.argtypes = [P, C.c_int64]
    L.pmf_run_set_batch_launch.argtypes = [P, C.c_int, C.c_int]
    L.pmf_run_get_batch_launch.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]
    L.pmf_run_batch_autotune.argtypes = [P, C.c_int64, _D]
    L.pmf_state_free_energy.argtypes = [P, _D, _D, _D, C.c_int]
    L.pmf_state_free_energy_from_samples.argtypes = [C.c_void_p, C.c_int, _D, C.c_int, C.c_int, _I64, C.c_double,
                                                     C.c_double, _D, _D, _D]
    L.pmf_free_energy_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64,
                                          C.c_double, C.c_double, C.c_void_p]
    L.pmf_mlp_create.argtypes = [_F, C.c_double, C.c_double, C.POINTER(P)]
    L.pmf_mlp_destroy.argtypes = [P]
    L.pmf_mlp_destroy.restype = None
    L.pmf_mlp_get_params.argtypes = [P, _F]
    L.pmf_mlp_predict.argtypes = [P, _D, C.c_int, _D, _D]
    L.pmf_mlp_gradient.argtypes = [P, _D, _F, C.c_int, _F, _D]
    L.pmf_mlp_train.argtypes = [P, P, C.c_int, C.c_int, C.c_double, C.c_uint64, _D]
    L.pmf_mlp_set_split.argtypes = [P, C.c_int]
    L.pmf_overlap.argtypes = [_D, _D, C.c_int, _D]
    L.pmf_run_adaptive.argtypes = [P, _D, C.c_int, C.POINTER(RunParams), C.POINTER(AdaptiveParams),
                                   C.POINTER(AdaptiveInfo), C.POINTER(FreeEnergyResult)]
    L.pmf_chain_set_warps.argtypes = [P, C.c_int, C.c_int]
    L.pmf_chain_set_grid.argtypes = [P, C.c_int, C.c_int, C.c_int]
    L.pmf_chain_get_launch.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.pmf_chain_set_schedule.argtypes = [P, C.c_int, C.c_int]
    L.pmf_chain_get_schedule.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
    L.pmf_chain_schedule_variants.restype = C.c_int
    L.pmf_chain_schedule_variant.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_size_t,
                                             C.POINTER(C.c_size_t), C.POINTER(C.c_int)]
    L.pmf_chain_autotune.argtypes = [P, _D, C.c_int, C.POINTER(RunParams), C.c_int, C.POINTER(C.c_int), _D]
    L.pmf_fp32_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D]
    L.pmf_fp64_peak.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D]
    L.pmf_set_stream.argtypes = [C.c_void_p]
    L.pmf_last_error.restype = C.c_char_p
    L.pmf_version.restype = C.c_char_p
    for name in ("pmf_create_system", "pmf_run_windows", "pmf_run_prepare", "pmf_run_prepare_seeded", "pmf_run_batch_prepare",
                 "pmf_run_prepare_sequential", "pmf_run_prepare_smd", "pmf_smd_work", "pmf_smd_free_energy",
                 "pmf_free_energy_item", "pmf_run_launch",
                 "pmf_run_wait", "pmf_get_run_info", "pmf_x_samples", "pmf_work_samples",
                 "pmf_free_energy", "pmf_free_energy_from_samples", "pmf_final_state",
                 "pmf_run_partials", "pmf_free_energy_from_partials", "pmf_work_distributions", "pmf_philox",
                 "pmf_chain_forces", "pmf_chain_schedule", "pmf_run_reduce", "pmf_run_set_queue_start", "pmf_run_set_batch_launch",
                 "pmf_run_get_batch_launch", "pmf_run_batch_autotune", "pmf_state_free_energy",
                 "pmf_state_free_energy_from_samples", "pmf_free_energy_noalloc",
                 "pmf_mlp_create", "pmf_mlp_get_params", "pmf_mlp_predict", "pmf_mlp_gradient", "pmf_mlp_train",
                 "pmf_overlap", "pmf_run_adaptive", "pmf_chain_set_warps", "pmf_chain_set_grid", "pmf_chain_get_launch",
                 "pmf_chain_set_schedule", "pmf_chain_get_schedule", "pmf_chain_schedule_variant",
                 "pmf_chain_autotune", "pmf_fp32_peak", "pmf_fp64_peak", "pmf_set_stream"):
        getattr(L, name).restype = C.c_int
    return L


lib = _load()


def _check(status, where):
    if status != PMF_OK:
        raise PmfError(status, where, lib.pmf_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(_D)


def pmf_version() -> str:
    return lib.pmf_version().decode()


def pmf_set_stream(stream_handle: int | None):
    """stream_handle: an integer cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)."""
    _check(lib.pmf_set_stream(C.c_void_p(stream_handle or 0)), "pmf_set_stream")


class System:
    """Owner of a pmf_system handle (and of the arrays passed to it)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib.pmf_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pmf_create_system_chain(chains, starts, precision=PMF_FP32) -> System:
    """chains: list of inputs.ChainParams (same bonded constants); starts: list of [N, 3]."""
    chains = list(chains)
    starts = list(starts)
    cat = lambda f: np.ascontiguousarray(np.concatenate([np.asarray(f(c), dtype=np.float64).ravel()
                                                          for c in chains]))
    keep = dict(n=np.array([c.n for c in chains], dtype=np.int32), sigma=cat(lambda c: c.sigma),
                eps=cat(lambda c: c.epsilon), q=cat(lambda c: c.charge), m=cat(lambda c: c.mass),
                dk=cat(lambda c: c.dih_k), dph=cat(lambda c: c.dih_phase),
                pos=np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.float64).ravel()
                                                         for s in starts])))
    c0 = chains[0]
    d = SystemDesc(model=PMF_MODEL_CHAIN, precision=precision, n_chains=len(chains),
                   n_beads=keep["n"].ctypes.data_as(C.POINTER(C.c_int)), sigma=_dp(keep["sigma"]),
                   epsilon=_dp(keep["eps"]), charge=_dp(keep["q"]), mass=_dp(keep["m"]),
                   dih_k=_dp(keep["dk"]), dih_phase=_dp(keep["dph"]), pos0=_dp(keep["pos"]),
                   bond_k=c0.kb, bond_r0=c0.r0, angle_k=c0.ktheta, angle_theta0=c0.theta0,
                   coulomb_k=c0.ke, nonbonded=int(c0.nonbonded))
    h = C.c_void_p()
    _check(lib.pmf_create_system(C.byref(d), C.byref(h)), "pmf_create_system")
    return System(h, keep)


def pmf_create_system_1d(a=2.0, x0=-1.0) -> System:
    d = SystemDesc(model=PMF_MODEL_1D_DOUBLEWELL, dw_a=a, x0=x0)
    h = C.c_void_p()
    _check(lib.pmf_create_system(C.byref(d), C.byref(h)), "pmf_create_system")
    return System(h, None)


def make_params(run, chain=0, n_steps_per_window=None, timeout_s=0.0, uid_base=0, segment_wait_s=0.0):
    """RunParams from an inputs.RunSettings."""
    arr = None
    if n_steps_per_window is not None:
        arr = np.ascontiguousarray(n_steps_per_window, dtype=np.int64)
    p = RunParams(k=run.k, kT=run.kT, dt=run.dt, gamma=run.gamma, n_steps=run.n_steps,
                  n_steps_per_window=arr.ctypes.data_as(_I64) if arr is not None else None,
                  n_equil=run.n_equil, sample_stride=run.stride, replicas=run.replicas,
                  seed=run.seed, uid_base=uid_base, chain=chain, timeout_s=timeout_s,
                  segment_wait_s=segment_wait_s)
    return p, arr


class Run:
    """Owner of a pmf_run handle."""

    def __init__(self, handle, lambdas, keep=None):
        self.handle = handle
        self.lambdas = np.asarray(lambdas, dtype=np.float64)
        self._keep = keep

    def close(self):
        if self.handle:
            lib.pmf_destroy_run(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch(self):
        _check(lib.pmf_run_launch(self.handle), "pmf_run_launch")

    def wait(self):
        _check(lib.pmf_run_wait(self.handle), "pmf_run_wait")

    def reduce(self):
        _check(lib.pmf_run_reduce(self.handle), "pmf_run_reduce")

    def set_batch_launch(self, mode, policy=0):
        """Batched runs: PMF_BATCH_PACKED (one persistent launch per chunk,
        packing policy 0, 1 or 2) or PMF_BATCH_GRAPH (per-item launches)."""
        _check(lib.pmf_run_set_batch_launch(self.handle, mode, policy), "pmf_run_set_batch_launch")

    def batch_launch(self):
        """dict(mode, policy, packs, ctas, teams[item]) of a batched run."""
        n = len(getattr(self, "item_windows", [1]))
        mode, pol, packs, ctas = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        teams = np.zeros(n, dtype=np.int32)
        _check(lib.pmf_run_get_batch_launch(self.handle, C.byref(mode), C.byref(pol), C.byref(packs), C.byref(ctas),
                                            teams.ctypes.data_as(C.POINTER(C.c_int)), n), "pmf_run_get_batch_launch")
        return dict(mode=mode.value, policy=pol.value, packs=packs.value, ctas=ctas.value, teams=teams)

    def batch_autotune(self, probe_steps=2000):
        """Time graph and packed launches of the batch (probe_steps each) and keep the fastest."""
        ms = C.c_double()
        _check(lib.pmf_run_batch_autotune(self.handle, int(probe_steps), C.byref(ms)), "pmf_run_batch_autotune")
        return ms.value

    def set_queue_start(self, first_item):
        """Test hook of the bounded device wait (pmf_run_set_queue_start)."""
        _check(lib.pmf_run_set_queue_start(self.handle, int(first_item)), "pmf_run_set_queue_start")

    def info(self):
        inf = RunInfo()
        _check(lib.pmf_get_run_info(self.handle, C.byref(inf)), "pmf_get_run_info")
        s = inf.n_windows
        return dict(n_windows=s, replicas=inf.replicas, total_samples=inf.total_samples,
                    samples_per_window=np.array(inf.samples_per_window[:s]),
                    sample_offset=np.array(inf.sample_offset[:s]))

    def x_samples(self):
        """Per-window arrays [R, T_w] (float32)."""
        inf = self.info()
        out = np.zeros(inf["total_samples"], dtype=np.float32)
        n = C.c_size_t()
        _check(lib.pmf_x_samples(self.handle, out.ctypes.data_as(_F), out.size, C.byref(n)), "pmf_x_samples")
        R = inf["replicas"]
        return [out[o:o + R * t].reshape(R, t) for o, t in
                zip(inf["sample_offset"], inf["samples_per_window"])]

    def work_samples(self, mode=PMF_WORK_PER_WINDOW_INCREMENT):
        n = C.c_size_t()
        lib.pmf_work_samples(self.handle, mode, None, 0, C.byref(n))
        out = np.zeros(n.value, dtype=np.float64)
        _check(lib.pmf_work_samples(self.handle, mode, _dp(out), out.size, C.byref(n)), "pmf_work_samples")
        return out

    def free_energy(self):
        return _fe_call(lambda res: lib.pmf_free_energy(self.handle, C.byref(res)), self.lambdas.size,
                        "pmf_free_energy")

    def free_energy_item(self, item, n_windows):
        return _fe_call(lambda res: lib.pmf_free_energy_item(self.handle, item, C.byref(res)), n_windows,
                        "pmf_free_energy_item")

    def work_distributions(self, x_lo, dx, n_x, dw, M, left_edge=False, with_omega=True):
        """App. C work distributions: dict with omega [s, 2M + 1] (if asked),
        dF_JE, var_ZW, lost."""
        s = self.lambdas.size
        hp = HistParams(x_lo, dx, n_x, dw, M, int(left_edge))
        om = np.zeros((s, 2 * M + 1)) if with_omega else None
        dF, var, lost = np.zeros(s), np.zeros(s), np.zeros(s)
        _check(lib.pmf_work_distributions(self.handle, C.byref(hp), _dp(om) if om is not None else None,
                                          om.size if om is not None else 0, _dp(dF), _dp(var), _dp(lost)),
               "pmf_work_distributions")
        return {"omega": om, "dF_JE": dF, "var_ZW": var, "lost": lost}

    def state_free_energy(self):
        """Eq. (15): dict with G and se_G per profile point and dF_turn_on (Eq. (5))."""
        s = self.lambdas.size
        G, se, on = np.zeros(s), np.zeros(s), C.c_double()
        _check(lib.pmf_state_free_energy(self.handle, _dp(G), _dp(se), C.byref(on), s), "pmf_state_free_energy")
        return {"G": G, "se_G": se, "dF_turn_on": on.value}

    def smd_work(self):
        """Accumulated work [replicas, records] of a pulled run."""
        n = C.c_size_t()
        lib.pmf_smd_work(self.handle, None, 0, C.byref(n))
        out = np.zeros(n.value)
        _check(lib.pmf_smd_work(self.handle, _dp(out), out.size, C.byref(n)), "pmf_smd_work")
        return out.reshape(self.info()["replicas"], -1)

    def smd_free_energy(self):
        T = int(self.info()["samples_per_window"][0])
        names = ("lambda", "dF_JE", "dF_cumulant", "W_mean", "W_var", "mean_x")
        arrs = {k: np.zeros(T) for k in names}
        _check(lib.pmf_smd_free_energy(self.handle, *[_dp(arrs[k]) for k in names], T), "pmf_smd_free_energy")
        return arrs

    def partials(self):
        """Per-replica partial sums [n_windows, replicas, 5] (pmf_run_partials)."""
        n = C.c_size_t()
        lib.pmf_run_partials(self.handle, None, 0, C.byref(n))
        out = np.zeros(n.value)
        _check(lib.pmf_run_partials(self.handle, _dp(out), out.size, C.byref(n)), "pmf_run_partials")
        return out.reshape(self.lambdas.size, -1, 5)

    def final_state(self):
        n = C.c_size_t()
        lib.pmf_final_state(self.handle, None, None, 0, C.byref(n))
        pos = np.zeros(n.value)
        vel = np.zeros(n.value)
        _check(lib.pmf_final_state(self.handle, _dp(pos), _dp(vel), n.value, C.byref(n)), "pmf_final_state")
        return pos, vel


def _fe_call(fn, s, where):
    arrs = {f: np.zeros(s) for f in RESULT_FIELDS}
    res = FreeEnergyResult(capacity=s, **{("lambda_" if f == "lambda" else f): _dp(a) for f, a in arrs.items()})
    _check(fn(res), where)
    return arrs


def pmf_run_prepare(system: System, lambdas, params) -> Run:
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    p, keep = params
    h = C.c_void_p()
    _check(lib.pmf_run_prepare(system.handle, _dp(lam), lam.size, C.byref(p), C.byref(h)), "pmf_run_prepare")
    return Run(h, lam, keep=(p, keep, system))


def pmf_run_prepare_sequential(system: System, lambdas, params) -> Run:
    """Sequential pulling protocol: params.replicas simulations each visit
    every window in order for params.n_steps steps."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    p, keep = params
    h = C.c_void_p()
    _check(lib.pmf_run_prepare_sequential(system.handle, _dp(lam), lam.size, C.byref(p), C.byref(h)),
           "pmf_run_prepare_sequential")
    return Run(h, lam, keep=(p, keep, system))


def pmf_run_prepare_smd(system: System, lambda1, velocity, params) -> Run:
    """Constant-velocity pulling: params.replicas simulations, the trap at
    lambda1 for params.n_equil steps, then advancing velocity * dt per step."""
    p, keep = params
    h = C.c_void_p()
    _check(lib.pmf_run_prepare_smd(system.handle, float(lambda1), float(velocity), C.byref(p), C.byref(h)),
           "pmf_run_prepare_smd")
    return Run(h, np.array([lambda1]), keep=(p, keep, system))


def pmf_run_prepare_seeded(system: System, lambdas, params, start) -> Run:
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    st = np.ascontiguousarray(start, dtype=np.float64)
    p, keep = params
    h = C.c_void_p()
    _check(lib.pmf_run_prepare_seeded(system.handle, _dp(lam), lam.size, C.byref(p), _dp(st), C.byref(h)),
           "pmf_run_prepare_seeded")
    return Run(h, lam, keep=(p, keep, system, st))


def pmf_run_batch_prepare(system: System, items, params) -> Run:
    """items: sequence of (chain index, lambda array); windows are laid end to
    end in item order.  The returned Run's lambdas are the concatenation and
    `item_windows` the per-item window counts."""
    lams = [np.ascontiguousarray(l, dtype=np.float64) for _, l in items]
    arr = (BatchItem * len(lams))(*[BatchItem(chain=int(c), n_windows=l.size, lambda_=_dp(l))
                                    for (c, _), l in zip(items, lams)])
    p, keep = params
    h = C.c_void_p()
    _check(lib.pmf_run_batch_prepare(system.handle, arr, len(lams), C.byref(p), C.byref(h)), "pmf_run_batch_prepare")
    run = Run(h, np.concatenate(lams), keep=(p, keep, system, lams, arr))
    run.item_windows = [l.size for l in lams]
    return run


def pmf_run_windows(system: System, lambdas, params) -> Run:
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    p, keep = params
    h = C.c_void_p()
    st = lib.pmf_run_windows(system.handle, _dp(lam), lam.size, C.byref(p), C.byref(h))
    run = Run(h, lam, keep=(p, keep, system)) if h.value else None
    if st != PMF_OK:
        err = PmfError(st, "pmf_run_windows", lib.pmf_last_error().decode())
        err.run = run
        raise err
    return run


def pmf_free_energy_from_partials(partials, lambdas, k, kT):
    """partials: [n_windows, replicas, 5] (shards concatenated on axis 1)."""
    P = np.ascontiguousarray(partials, dtype=np.float64)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    return _fe_call(lambda res: lib.pmf_free_energy_from_partials(_dp(P), _dp(lam), lam.size, P.shape[1], k, kT,
                                                                  C.byref(res)), lam.size,
                    "pmf_free_energy_from_partials")


def pmf_free_energy_from_samples(x, lambdas, replicas, samples_per_window, k, kT, x_on_device=False):
    """x: host float32 array in run layout, or (x_on_device=True) an integer device pointer."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    spw = np.ascontiguousarray(samples_per_window, dtype=np.int64)
    if x_on_device:
        xp = C.c_void_p(int(x))
    else:
        xa = np.ascontiguousarray(x, dtype=np.float32)
        xp = xa.ctypes.data_as(C.c_void_p)
    return _fe_call(lambda res: lib.pmf_free_energy_from_samples(xp, int(bool(x_on_device)), _dp(lam), lam.size,
                                                                 replicas, spw.ctypes.data_as(_I64), k, kT,
                                                                 C.byref(res)),
                    lam.size, "pmf_free_energy_from_samples")


def pmf_state_free_energy_from_samples(x, lambdas, replicas, samples_per_window, k, kT, x_on_device=False):
    """Eq. (15) on caller samples (layout of pmf_free_energy_from_samples)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    spw = np.ascontiguousarray(samples_per_window, dtype=np.int64)
    if x_on_device:
        xp = C.c_void_p(int(x))
    else:
        xa = np.ascontiguousarray(x, dtype=np.float32)
        xp = xa.ctypes.data_as(C.c_void_p)
    G, se, on = np.zeros(lam.size), np.zeros(lam.size), C.c_double()
    _check(lib.pmf_state_free_energy_from_samples(xp, int(bool(x_on_device)), _dp(lam), lam.size, replicas,
                                                  spw.ctypes.data_as(_I64), k, kT, _dp(G), _dp(se), C.byref(on)),
           "pmf_state_free_energy_from_samples")
    return {"G": G, "se_G": se, "dF_turn_on": on.value}


def pmf_philox(seed, c0, c1, c2, c3, n_blocks):
    raw = np.zeros((n_blocks, 4), dtype=np.uint32)
    nor = np.zeros((n_blocks, 4), dtype=np.float32)
    _check(lib.pmf_philox(seed, c0, c1, c2, c3, n_blocks, raw.ctypes.data_as(C.POINTER(C.c_uint32)),
                          nor.ctypes.data_as(_F)), "pmf_philox")
    return raw, nor


def pmf_chain_forces(system: System, chain, pos, lam, k):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    f = np.zeros_like(pos)
    _check(lib.pmf_chain_forces(system.handle, chain, _dp(pos), lam, k, _dp(f)), "pmf_chain_forces")
    return f


def pmf_chain_schedule(N, NW=4, precision=PMF_FP32, variant=0):
    """Host schedule: int array [pieces, 7] (warp, I1, I2, J, kind, near1, near2), padded N."""
    n = C.c_size_t()
    pad = C.c_int()
    lib.pmf_chain_schedule_variant(N, NW, precision, variant, None, 0, C.byref(n), C.byref(pad))
    out = np.zeros(7 * n.value, dtype=np.int32)
    _check(lib.pmf_chain_schedule_variant(N, NW, precision, variant, out.ctypes.data_as(C.POINTER(C.c_int)),
                                          out.size, C.byref(n), C.byref(pad)), "pmf_chain_schedule_variant")
    return out.reshape(-1, 7), pad.value


def pmf_chain_schedule_variants():
    return lib.pmf_chain_schedule_variants()


def pmf_chain_set_schedule(system: System, chain, variant):
    _check(lib.pmf_chain_set_schedule(system.handle, chain, variant), "pmf_chain_set_schedule")


def pmf_chain_get_schedule(system: System, chain=0):
    v = C.c_int()
    _check(lib.pmf_chain_get_schedule(system.handle, chain, C.byref(v)), "pmf_chain_get_schedule")
    return v.value


def pmf_free_energy_noalloc(x_dev, lambda_dev, n_windows, replicas, samples_per_window, k, kT, out_dev):
    """Allocation-free reduction; every pointer is an integer device address.
    out_dev receives 14 * n_windows doubles (RESULT_FIELDS order).  Returns
    after enqueueing on the library stream."""
    _check(lib.pmf_free_energy_noalloc(C.c_void_p(int(x_dev)), C.c_void_p(int(lambda_dev)), n_windows,
                                       replicas, samples_per_window, k, kT, C.c_void_p(int(out_dev))),
           "pmf_free_energy_noalloc")


PMF_MLP_PARAMS = 4418


def pack_mlp_params(p) -> np.ndarray:
    """FP32 packing W1[64], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).ravel()
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


class Mlp:
    """Owner of a pmf_mlp handle (surrogate lambda -> mean / log-variance of x)."""

    def __init__(self, params, c, h):
        w = np.ascontiguousarray(params, dtype=np.float32)
        if w.size != PMF_MLP_PARAMS:
            raise ValueError("need PMF_MLP_PARAMS weights")
        self.handle = C.c_void_p()
        _check(lib.pmf_mlp_create(w.ctypes.data_as(_F), c, h, C.byref(self.handle)), "pmf_mlp_create")

    def close(self):
        if self.handle:
            lib.pmf_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.zeros(PMF_MLP_PARAMS, dtype=np.float32)
        _check(lib.pmf_mlp_get_params(self.handle, out.ctypes.data_as(_F)), "pmf_mlp_get_params")
        return out

    def predict(self, lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        mu = np.zeros_like(lam)
        lv = np.zeros_like(lam)
        _check(lib.pmf_mlp_predict(self.handle, _dp(lam), lam.size, _dp(mu), _dp(lv)), "pmf_mlp_predict")
        return mu, lv

    def gradient(self, lam, x):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float32)
        g = np.zeros(PMF_MLP_PARAMS, dtype=np.float32)
        loss = C.c_double()
        _check(lib.pmf_mlp_gradient(self.handle, _dp(lam), x.ctypes.data_as(_F), lam.size, g.ctypes.data_as(_F),
                                    C.byref(loss)), "pmf_mlp_gradient")
        return g, loss.value

    def set_split(self, split):
        _check(lib.pmf_mlp_set_split(self.handle, int(split)), "pmf_mlp_set_split")

    def train(self, run, steps, batch, lr, seed):
        loss = C.c_double()
        _check(lib.pmf_mlp_train(self.handle, run.handle, steps, batch, lr, seed, C.byref(loss)), "pmf_mlp_train")
        return loss.value


def pmf_overlap(mu, log_var):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    lv = np.ascontiguousarray(log_var, dtype=np.float64)
    out = np.zeros(mu.size - 1)
    _check(lib.pmf_overlap(_dp(mu), _dp(lv), mu.size, _dp(out)), "pmf_overlap")
    return out


def pmf_run_adaptive(system: System, lambda0, params, mlp_init, threshold=0.3, max_rounds=3, max_windows=64,
                     mlp_steps=300, mlp_batch=512, mlp_lr=3e-3, mlp_seed=1, trace=False, continue_windows=False,
                     train_on_gap=False):
    """Surrogate-guided window insertion; returns (info dict, free-energy dict).
    With trace=True the info dict also holds "trace": one dict per round with
    the decisions of pmf_adaptive_trace (windows, predictions, overlaps,
    inserted centres, seeding targets, candidates' final x, the candidate
    each replica of an inserted window started from, whether the round
    trained and, with train_on_gap, the measured overlaps)."""
    lam = np.ascontiguousarray(lambda0, dtype=np.float64)
    w = np.ascontiguousarray(mlp_init, dtype=np.float32)
    p, keep = params
    tr = None
    if trace:
        R, Q, W = p.replicas, max(max_rounds, 1), max_windows
        ta = dict(n_windows=np.zeros(Q, np.int32), n_inserted=np.zeros(Q, np.int32), lambda_=np.zeros((Q, W)),
                  mu=np.zeros((Q, W)), log_var=np.zeros((Q, W)), ovl=np.zeros((Q, W)), inserted=np.zeros((Q, W)),
                  target=np.zeros((Q, W)), cand_x=np.zeros((Q, W, 2 * R)), seed=np.zeros((Q, W, R), np.int32),
                  data_ovl=np.full((Q, W), np.nan), trained=np.full(Q, -1, np.int32))
        tr = AdaptiveTrace(max_rounds=Q, max_windows=W, replicas=R, rounds=0,
                           **{k: (a.ctypes.data_as(_IP) if a.dtype == np.int32 else _dp(a)) for k, a in ta.items()})
    ap = AdaptiveParams(threshold, max_rounds, max_windows, mlp_steps, mlp_batch, mlp_lr, mlp_seed,
                        w.ctypes.data_as(_F), C.pointer(tr) if tr is not None else None, int(bool(continue_windows)),
                        int(bool(train_on_gap)))
    info = AdaptiveInfo()
    res_arrays = {f: np.zeros(max_windows) for f in RESULT_FIELDS}
    res = FreeEnergyResult(capacity=max_windows,
                           **{("lambda_" if f == "lambda" else f): _dp(a) for f, a in res_arrays.items()})
    _check(lib.pmf_run_adaptive(system.handle, _dp(lam), lam.size, C.byref(p), C.byref(ap), C.byref(info),
                                C.byref(res)), "pmf_run_adaptive")
    n = info.n_windows
    out = {f: a[:n].copy() for f, a in res_arrays.items()}
    meta = dict(n_windows=n, rounds=info.rounds, inserted=info.inserted, gpu_seconds=info.gpu_seconds,
                mlp_loss=info.mlp_loss, lambdas=np.array(info.lambda_[:n]))
    if tr is not None:
        rounds = []
        for q in range(tr.rounds):
            nw, ni = int(ta["n_windows"][q]), int(ta["n_inserted"][q])
            rounds.append(dict(lambdas=ta["lambda_"][q, :nw].copy(), mu=ta["mu"][q, :nw].copy(),
                               log_var=ta["log_var"][q, :nw].copy(), ovl=ta["ovl"][q, :max(nw - 1, 0)].copy(),
                               inserted=ta["inserted"][q, :ni].copy(), target=ta["target"][q, :ni].copy(),
                               cand_x=ta["cand_x"][q, :ni].copy(), seed=ta["seed"][q, :ni].copy(),
                               trained=int(ta["trained"][q]), data_ovl=ta["data_ovl"][q, :max(nw - 1, 0)].copy()))
        meta["trace"] = rounds
    return meta, out


def pmf_chain_set_warps(system: System, chain, warps):
    _check(lib.pmf_chain_set_warps(system.handle, chain, warps), "pmf_chain_set_warps")


def pmf_chain_set_grid(system: System, chain, ctas, seg_steps=0):
    _check(lib.pmf_chain_set_grid(system.handle, chain, ctas, seg_steps), "pmf_chain_set_grid")


def pmf_chain_get_launch(system: System, chain=0):
    """(warps, ctas, seg_steps) of a chain's launch shape."""
    w, c, g = C.c_int(), C.c_int(), C.c_int()
    _check(lib.pmf_chain_get_launch(system.handle, chain, C.byref(w), C.byref(c), C.byref(g)), "pmf_chain_get_launch")
    return w.value, c.value, g.value


def pmf_fp32_peak(packed=True, ctas_per_sm=0, iters=1 << 16, reps=3):
    """Measured FP32 FMA throughput of the GPU in TFLOP/s (FMA = 2 flops)
    and the time of the best launch in ms."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib.pmf_fp32_peak(int(bool(packed)), ctas_per_sm, iters, reps, C.byref(tf), C.byref(ms)), "pmf_fp32_peak")
    return tf.value, ms.value


def pmf_fp64_peak(ctas_per_sm=0, iters=1 << 12, reps=3):
    """Measured FP64 FMA throughput in TFLOP/s (FMA = 2 flops) and the time
    of the best launch in ms."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib.pmf_fp64_peak(ctas_per_sm, iters, reps, C.byref(tf), C.byref(ms)), "pmf_fp64_peak")
    return tf.value, ms.value


def pmf_chain_autotune(system: System, lambdas, params, probe_steps=400):
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    p, keep = params
    best = C.c_int()
    ms = C.c_double()
    _check(lib.pmf_chain_autotune(system.handle, _dp(lam), lam.size, C.byref(p), probe_steps, C.byref(best),
                                  C.byref(ms)), "pmf_chain_autotune")
    return best.value, ms.value
