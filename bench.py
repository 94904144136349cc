"""Benchmark of the coupled IBM-LBM time step on GB300.

Default workload (N = 1): 256^3 D3Q19 lattice, tube of radius 120 along x
with bounce-back walls, body-force drive (centreline Re ~ 1), 3000
biconcave red-cell membranes of 642 vertices (diameter 16 lu), FP32
population storage. One "step" = one coupled time step (marker forces,
spreading, collide-stream, interpolation + advection).

Prints ONE JSON line (rank 0):
  value        lattice updates per second over the whole box (MLUPS), inputs
               resident in HBM, device time (CUDA events), max over ranks
  e2e          same metric through the C ABI with host buffers: upload of the
               lattice state and markers, K steps, download of fields and
               markers inside the timed region
  roofline     the collide-stream kernel (the dominant one): algorithmic bytes
               per launch / its average event-timed duration, against the
               measured HBM copy bandwidth
  cpu_baseline the FP64 oracle as it stands, one full coupled step of the
               same workload on one host core
With --gpus N > 1 (launched under torchrun) every rank runs an independent
replica of the workload on its own GPU: the path has no exchange step, so
there is no collective on the data path ("scaling": "weak").
``--impl reference`` times the oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = 'coupled IBM-LBM MLUPS & % of HBM roofline (1 GB300); batched p50/p99 latency'
UNIT = 'MLUPS'


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def make_workload(name: str):
    from paper_1704_04551_gb300 import inputs as I
    if name in ('tube256', 'tube256_f16', 'tube256_bf16'):
        w = I.rbc_tube(n=256, radius=120.0, n_cells=3000, seed=1706, steps=2000)
        w['storage'] = {'tube256': 'f32', 'tube256_f16': 'f16', 'tube256_bf16': 'bf16'}[name]
        w['label'] = f'rbc_tube_256^3_R120_3000x642_{w["storage"]}'
        return w
    if name == 'tube160':
        # same cell density and Re as the 256^3 case, for detailed profiles
        w = I.rbc_tube(n=160, radius=75.0, n_cells=732, seed=1706, steps=200)
        w['storage'] = 'f32'
        w['label'] = 'rbc_tube_160^3_R75_732x642_f32'
        return w
    if name == 'tube64':
        w = I.rbc_tube(n=64, radius=30.0, n_cells=50, seed=1707, steps=1000)
        w['storage'] = 'f32'
        w['label'] = 'rbc_tube_64^3_R30_50x642_f32'
        return w
    if name in ('mix512', 'mix512_f32'):
        # red cells and filaments in a channel with Morse excluded volume
        w = I.mixed_suspension(shape=(512, 512, 512), n_cells=20000, n_filaments=4000, beads=50, seed=1709,
                               steps=1000)
        w['storage'] = 'f16' if name == 'mix512' else 'f32'
        w['label'] = f'mixed_channel_512^3_20000x642_cells_4000x50_filaments_{w["storage"]}'
        return w
    if name == 'mix128':
        # 128 x 64 x 64 copy of the mixed suspension at the same cell and filament densities
        w = I.mixed_suspension(shape=(128, 64, 64), n_cells=39, n_filaments=16, beads=50, seed=1709, steps=1000)
        w['storage'] = 'f16'
        w['label'] = 'mixed_channel_128x64x64_39x642_cells_16x50_filaments_f16'
        return w
    if name == 'serve':
        # the first case of the serving stream (the reference arm's sample)
        w = I.serving_stream(n_cases=1, seed=1708)[0]
        w['storage'] = 'f32'
        w['label'] = 'serving_stream_case0_' + w['name']
        return w
    if name == 'shear32':
        w = I.shear_ellipsoid(n=32, steps=500)
        w['storage'] = 'f32'
        w['label'] = 'rigid_ellipsoid_shear_32^3_f32'
        return w
    raise ValueError(name)


def fluid_cells(lat):
    nx, ny, nz = lat['nx'], lat['ny'], lat['nz']
    if lat['geometry'] != 2:
        return nx * ny * nz
    y, z = np.meshgrid(np.arange(ny), np.arange(nz), indexing='ij')
    yc, zc = (ny - 1) / 2, (nz - 1) / 2
    R2 = np.float32(lat['tube_radius'] ** 2)
    dy = (y - yc).astype(np.float32)
    dz = (z - zc).astype(np.float32)
    return int(nx * np.count_nonzero(~(dy * dy + dz * dz > R2)))


def touched_cells(lat, X):
    """Fluid cells inside the 4^3 delta stencil of at least one marker."""
    nx, ny, nz = lat['nx'], lat['ny'], lat['nz']
    mask = np.zeros((nz, ny, nx), dtype=bool)
    base = np.floor(X).astype(np.int64) - 1
    for c in range(4):
        z = base[2] + c
        for b in range(4):
            y = base[1] + b
            for a in range(4):
                x = np.mod(base[0] + a, nx)
                if lat['geometry'] == 0:
                    yy, zz, ok = np.mod(y, ny), np.mod(z, nz), slice(None)
                    mask[zz, yy, x] = True
                    continue
                if lat['geometry'] == 1:
                    zz = np.mod(z, nz)
                    ok = (y >= 0) & (y < ny)
                    mask[zz[ok], y[ok], x[ok]] = True
                else:
                    ok = (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
                    mask[z[ok], y[ok], x[ok]] = True
    if lat['geometry'] == 2:
        zz, yy = np.meshgrid(np.arange(nz), np.arange(ny), indexing='ij')
        dy = (yy - (ny - 1) / 2).astype(np.float32)
        dz = (zz - (nz - 1) / 2).astype(np.float32)
        solid = dy * dy + dz * dz > np.float32(lat['tube_radius'] ** 2)
        mask &= ~solid[:, :, None]
    return int(mask.sum())


def bytes_per_pop(storage):
    return 4 if storage == 'f32' else 2


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.dev), f'--query-gpu={self.Q}',
                                          '--format=csv,noheader,nounits', '-lms', '100'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['nvidia-smi unavailable'], samples=0)
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for line in self.lines:
            parts = [p.strip() for p in line.split(',')]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == 'active':
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def measured_peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d['hbm_gbs']), 'measured'
    return 6800.0, 'fallback'


def source_sha(names):
    """Hash of the code of the given csrc files, comments and blank lines
    removed (a comment edit does not change the kernel the counters were
    taken on)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, 'paper_1704_04551_gb300', 'csrc', name)) as f:
            for line in f:
                code = line.split('//', 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b'\n')
    return h.hexdigest()[:16]


def collide_source_sha():
    """Hash of the sources the collide kernel is built from."""
    return source_sha(('common.cuh', 'lbm_cell.cuh', 'lbm.cu'))


def couple_source_sha():
    """Hash of the sources the fused coupling kernel is built from."""
    return source_sha(('common.cuh', 'transfer_group.cuh', 'forces_body.cuh', 'couple.cu'))


def couple_traffic(bodies):
    """DRAM bytes per fused coupling launch: the committed ncu summary's
    bytes per body times the bodies, if the kernel source is unchanged since
    the capture."""
    p = os.path.join(ROOT, 'profiles', 'couple_tube160_f32.md')
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ':' in line and line.startswith('- '):
            k, v = line[2:].split(':', 1)
            vals[k.strip()] = v.strip().strip('`')
    if vals.get('couple source sha256 prefix') != couple_source_sha():
        return None
    try:
        return float(vals['dram bytes per body']) * bodies
    except (KeyError, ValueError):
        return None


def collide_traffic(storage, workload):
    """DRAM bytes per collide launch of the 256^3 tube from the committed ncu
    summary, if the kernel source is unchanged since it was taken (other
    workloads: None, their force-density share differs)."""
    if not workload.startswith('tube256'):
        return None
    sha = collide_source_sha()
    p = os.path.join(ROOT, 'profiles', f'collide_tube256_{storage}.md')
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ':' in line and line.startswith('- '):
            k, v = line[2:].split(':', 1)
            vals[k.strip()] = v.strip().strip('`')
    if vals.get('collide source sha256 prefix') != sha:
        return None
    try:
        return float(vals['dram bytes per launch (full size)'])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------
# distributed helpers (replicas only)
# ----------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault('MASTER_ADDR', '127.0.0.1')
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def reduce_max(dist, value, device='cpu'):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(units_per_rank, max_seconds, n_ranks):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    return units_per_rank * n_ranks / max_seconds


# ----------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle as it stands
# ----------------------------------------------------------------------------
def host_cpu():
    """Host cores and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(['lscpu'], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith('Model name:'):
                model = line.split(':', 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open('/proc/cpuinfo'):
                if line.startswith('model name'):
                    model = line.split(':', 1)[1].strip()
                    break
        except OSError:
            pass
    return dict(nproc=os.cpu_count(), model=model or 'unknown')


def time_oracle(w, steps, warmup=0, threads=0):
    """The FP64 oracle on `threads` host threads (0: all of them)."""
    import oracle as O
    O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    t0 = time.perf_counter()
    o = O.Oracle.from_workload(w)
    setup = time.perf_counter() - t0
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    N = w['lattice']['nx'] * w['lattice']['ny'] * w['lattice']['nz']
    return dict(mlups=N * steps / dt / 1e6, seconds=dt, setup_s=setup, steps=steps, threads=O.set_threads(0))


def cpu_sample(name):
    """The workload the FP64 oracle is timed on: the workload itself, or a
    bounded copy where one oracle step would not finish in seconds (the
    oracle's Morse term visits every pair of markers)."""
    if name in ('mix512', 'mix512_f32'):
        return make_workload('mix128')
    return make_workload(name)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = cpu_sample(args.workload)
    # each requested step is bounded: at most a couple of full oracle steps
    # are timed, after at most three untimed ones, so that the whole run ends
    # within a few minutes
    n = max(1, min(args.steps, args.ref_max_steps))
    wu = max(0, min(args.warmup, 3))
    r = time_oracle(w, n, warmup=wu)
    cpu = host_cpu()
    line = dict(impl='reference', metric=METRIC, value=r['mlups'], unit=UNIT, n_gpus=args.gpus, steps=n,
                warmup=wu, ms_per_step=1e3 * r['seconds'] / n, higher_is_better=True, scaling='weak',
                vs_baseline=None, dtype='f64', data='synthetic',
                config=dict(workload=w['label'], requested_steps=args.steps, lattice=[w['lattice'][k] for k in ('nx', 'ny', 'nz')],
                            markers=int(w['X'].shape[1]), bodies=len(w['bodies'])),
                cpu_baseline=dict(value=r['mlups'], unit=UNIT, cores=r['threads'], kind='oracle',
                                  sample=f'{n} full coupled step(s) of {w["label"]} on {r["threads"]} host threads '
                                         f'(FP64 C oracle, OpenMP over its independent loops)',
                                  nproc=cpu['nproc'], cpu_model=cpu['model']),
                e2e=dict(value=r['mlups'], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def kernels_per_step(w):
    """Kernels of the library launched per coupled step of workload w:
    marker forces (membranes, rigid bodies, filaments, and the ten of the
    Morse neighbour lists), spreading, collide, interpolation."""
    kinds = {b['kind'] for b in w['bodies']}
    n = 1  # collide
    if w['X'].shape[1] > 0:
        n += 2  # spreading, interpolation
        n += int(0 in kinds) + int(bool(kinds & {1, 3})) + int(2 in kinds)
        if (w.get('morse') or {}).get('rc', 0) > 0:
            n += 10
    return n


def production_launches(w, steps, fused):
    """Kernels ibm_lbm_step launches for `steps` steps from an even AA step:
    fused chunks of 64 (while more than 64 steps remain) or 16 steps (first
    step's forces and spreading, then collide + fused kernel per step, the
    last interpolation alone), the remaining steps one by one through the
    separate kernels, and the conservation check. Without the fused path
    every step takes the separate kernels."""
    per_step = kernels_per_step(w)
    if not fused:
        return per_step * steps + 1
    n, left = 0, steps
    while left > 16:
        c = 64 if left > 64 else 16
        n += 2 + c + (c - 1) + 1
        left -= c
    return n + per_step * left + 1


def fused_path(w, storage):
    """Whether ibm_lbm_step takes the fused coupling kernel for workload w:
    every marker in a membrane body, no Morse term (the library decides the
    same at set_markers / step time)."""
    bodies = w['bodies']
    if not bodies or (w.get('morse') or {}).get('rc', 0) > 0:
        return False
    if any(b['kind'] != 0 for b in bodies):
        return False
    # templates of up to ~938 vertices (the fused kernel's shared memory); the
    # production-path timing run confirms what the library chose
    return sum(b['count'] for b in bodies) == w['X'].shape[1] and w['mesh']['rest_X'].shape[1] <= 938


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    assert ws == args.gpus, f'--gpus {args.gpus} but WORLD_SIZE {ws}'
    torch.cuda.set_device(local)
    device = torch.device('cuda', local)
    dist = init_dist(ws, 'nccl')
    from paper_1704_04551_gb300 import binding, build
    build.build()
    w = make_workload(args.workload)
    storage = args.storage or w['storage']
    lat = w['lattice']
    N = lat['nx'] * lat['ny'] * lat['nz']
    Nf = fluid_cells(lat)
    M = int(w['X'].shape[1])

    sim = binding.Simulation.from_workload(w, storage=storage, device=local)
    stream = torch.cuda.ExternalStream(sim.stream, device=device)
    sim.step(args.warmup)

    # ---- timed region: K steps through the production launch path (CUDA
    # graphs of 16 steps, captured during the warm-up), inputs resident in HBM
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    sim.step_async(args.steps)
    end.record(stream)
    sim.synchronize()
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    barrier(dist, device)
    ms = start.elapsed_time(end)
    ms_max = reduce_max(dist, ms, device)
    diag = sim.diagnostics()
    # the same K steps again with an event around every stage (per-stage
    # split and the collide roofline; launched from the host, slightly slower)
    sim.set_timing(args.steps)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    s0.record(stream)
    sim.step_async(args.steps)
    s1.record(stream)
    sim.synchronize()
    staged_ms = s0.elapsed_time(s1)
    stages = sim.timing()
    sim.set_timing(0)
    value = aggregate(N * args.steps, ms_max / 1e3, ws) / 1e6
    # the same K steps on the production path with events around the
    # collision and the fused coupling kernel of every step that launches it
    # (membrane suspensions; other handles report per-stage times here)
    fused = fused_path(w, storage)
    prod = None
    if fused:
        sim.set_timing(args.steps, fused=True)
        sim.step(args.steps)
        prod = sim.timing()
        sim.set_timing(0)
        if not (prod['steps'] > 0 and prod['forces_ms'] == 0.0 and prod['spread_ms'] == 0.0):
            fused, prod = False, None

    # ---- rooflines: the collide-stream kernel, the fused coupling kernel and
    # the whole step. Algorithmic bytes per unit: N_f*38*s_p + N_touch*24 for
    # the collision (populations read and written once; force density read
    # and velocity written on touched cells), M*72 for the coupling (FP64 X
    # read and written, FP32 U and F handed off per marker). Launch durations
    # from CUDA events on the library's stream: the production-path timing
    # run for membrane suspensions, the per-stage run otherwise.
    sp = bytes_per_pop(storage)
    n_touch = touched_cells(lat, w['X'])
    alg_bytes = Nf * 38 * sp + n_touch * 24
    t = prod if prod is not None else stages
    collide_s = t['collide_ms'] / 1e3 / max(1, t['steps'])
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / collide_s / 1e9
    step_alg = alg_bytes + M * 72
    step_s = ms_max / 1e3 / args.steps
    collide = dict(kernel='k_collide (fused collide-stream-force)', bound='hbm', achieved=achieved, peak=peak,
                   unit='GB/s', frac=achieved / peak, traffic=collide_traffic(storage, args.workload),
                   alg_bytes_per_launch=alg_bytes, launch_ms=collide_s * 1e3)
    step = dict(step_alg_bytes=step_alg,
                step_alg_bytes_formula='N_f*38*s_p + N_touch*24 + M*72 (populations read+written once, force '
                                       'density read and velocity written on touched cells, FP64 X read+written '
                                       'and FP32 U, F per marker)',
                step_achieved=step_alg / step_s / 1e9,
                step_frac=(step_alg / step_s / 1e9) / peak)
    if prod is not None:
        # the fused coupling kernel takes the larger share of the step
        couple_s = prod['interp_ms'] / 1e3 / prod['steps']
        c_bytes = M * 72
        c_ach = c_bytes / couple_s / 1e9
        roof = dict(bound='hbm', achieved=c_ach, peak=peak, unit='GB/s', frac=c_ach / peak,
                    traffic=couple_traffic(len(w['bodies'])),
                    kernel='k_couple (fused: interpolation + advection, membrane forces, spreading of the next step)',
                    alg_bytes_per_launch=c_bytes, alg_bytes_formula='M*72', launch_ms=couple_s * 1e3,
                    note='latency-bound (see profiles/couple_tube160_f32.md); the HBM-bound kernel is `collide`',
                    peak_source=f'{peak_kind} hbm_gbs (burst copy)', collide=collide, **step)
    else:
        roof = dict(collide, peak_source=f'{peak_kind} hbm_gbs (burst copy)', **step)

    # ---- end to end through the C ABI with host buffers ----------------------
    rho0 = np.ones(N)
    u0 = np.zeros((3, N))
    X0 = np.ascontiguousarray(w['X'])
    rho_out = np.empty(N)
    u_out = np.empty((3, N))
    Xo, Uo, Fo = np.empty((3, M)), np.empty((3, M)), np.empty((3, M))
    barrier(dist, device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    binding.ibm_lbm_set_lattice(sim.h, rho0, u0)
    sim.set_markers(w.get('mesh'), w['bodies'], X0)
    binding.ibm_lbm_step(sim.h, args.steps)
    binding.ibm_lbm_get_fields(sim.h, rho_out, u_out)
    binding.ibm_lbm_get_markers(sim.h, Xo, Uo, Fo)
    e2e_s = reduce_max(dist, time.perf_counter() - t0, device)
    h2d = rho0.nbytes + u0.nbytes + X0.nbytes
    d2h = rho_out.nbytes + u_out.nbytes + Xo.nbytes + Uo.nbytes + Fo.nbytes
    e2e = dict(value=aggregate(N * args.steps, e2e_s, ws) / 1e6, unit=UNIT,
               h2d_bytes_per_step=h2d / args.steps, d2h_bytes_per_step=d2h / args.steps,
               note='one job: upload lattice state + markers, K steps, download fields + markers; bytes/step = job bytes / K')

    # ---- CPU baseline (rank 0, N = 1 only) -----------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ws_cpu = cpu_sample(args.workload)
        r = time_oracle(ws_cpu, 1)
        r1 = time_oracle(ws_cpu, 1, threads=1)
        hc = host_cpu()
        cpu = dict(value=r['mlups'], unit=UNIT, cores=r['threads'], kind='oracle',
                   sample=f'1 full coupled step of {ws_cpu["label"]} (FP64 C oracle, {r["threads"]} threads, '
                          f'setup excluded)',
                   seconds=r['seconds'], single_thread=dict(value=r1['mlups'], unit=UNIT, seconds=r1['seconds']),
                   nproc=hc['nproc'], cpu_model=hc['model'])

    if rank == 0:
        tot = sum(stages[k] for k in ('forces_ms', 'spread_ms', 'collide_ms', 'interp_ms'))
        split = {k: stages[k] / max(1, stages['steps']) for k in ('forces_ms', 'spread_ms', 'collide_ms', 'interp_ms')}
        half = max(1, stages['steps']) / 2
        split['collide_even_ms'] = (stages['collide_ms'] - stages['collide_odd_ms']) / half
        split['collide_odd_ms'] = stages['collide_odd_ms'] / half
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms_max / args.steps, higher_is_better=True, scaling='weak', vs_baseline=None,
            dtype='f32' if storage == 'f32' else f'f32 ({storage}-deviation storage)', data='synthetic',
            config=dict(workload=w['label'], lattice=[lat['nx'], lat['ny'], lat['nz']], fluid_cells=Nf,
                        touched_cells=n_touch, markers=M, bodies=len(w['bodies']), tau=lat['tau'],
                        filaments=sum(1 for b in w['bodies'] if b['kind'] == 2), morse=w.get('morse'),
                        body_force=lat['body_force'][0], storage=storage, seed=w['seed'],
                        mflups_fluid=Nf * args.steps * ws / (ms_max / 1e3) / 1e6,
                        production_path='collide + fused coupling kernel per step (membrane suspension)' if fused
                        else 'separate kernels per stage',
                        coupling_ms_per_step=ms_max / args.steps - split['collide_ms'],
                        production_ms_per_launch=None if prod is None else dict(
                            collide_ms=prod['collide_ms'] / prod['steps'], couple_ms=prod['interp_ms'] / prod['steps'],
                            steps_timed=prod['steps'],
                            note='events around each collision and each fused coupling kernel, direct launches'),
                        staged_path_ms_per_step=staged_ms / args.steps,
                        stage_ms_per_step=split,
                        coupling_share=(split['spread_ms'] + split['interp_ms']) / max(1e-12, tot / max(1, stages['steps'])),
                        l2='inputs larger than L2 (populations %.2f GB)' % (19 * N * sp / 1e9),
                        parallelism=f'replicas x{ws}' if ws > 1 else 'single GPU'),
            roofline=roof, cpu_baseline=cpu, e2e=e2e,
            clocks=dict(sm_mhz=clk['sm_mhz'], sm_max_mhz=clk['sm_max_mhz'], reasons=clk['reasons'],
                        samples=clk['samples']),
            gpu_launches=production_launches(w, args.steps, fused),
            diagnostics=dict(mass=diag['mass'], fluid_cells=diag['fluid_cells'], umax=diag['umax']),
            timed_stage_total_ms=tot)
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# serving: continuous batching of independent shear-cell cases
# ----------------------------------------------------------------------------
def serving_cases(args):
    from paper_1704_04551_gb300 import inputs as I
    cases = I.serving_stream(n_cases=args.serve_cases, seed=1708, periods=2.0, period_scale=args.period_scale)
    for w in cases:
        lat = w['lattice']
        w['N'] = lat['nx'] * lat['ny'] * lat['nz']
        w['B_step'] = w['N'] * 38 * 4 + touched_cells(lat, w['X']) * 24 + w['X'].shape[1] * 72
    return cases


def serve_batched(binding, cases, arrivals, args, keep=()):
    """Run the stream through one server; cases are submitted when their
    arrival time (seconds after the start) has passed. Returns per-case
    completion times, the number of chunks and the results of `keep`."""
    srv = binding.Server(args.serve_budget_gb * 1e9, max_active=args.serve_slots, chunk_steps=args.serve_chunk)
    n = len(cases)
    order = sorted(range(n), key=lambda i: arrivals[i])
    done_t, results, outstanding = [None] * n, {}, {}
    nxt, chunks, unstable = 0, 0, 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[order[nxt]] <= now:
            i = order[nxt]
            outstanding[srv.submit(cases[i], cases[i]['steps'])] = i
            nxt += 1
        if not outstanding:
            if nxt == n:
                break
            time.sleep(max(0.0, arrivals[order[nxt]] - now))
            continue
        rc, running, pending, _ = srv.advance()
        chunks += 1
        unstable += rc != binding.OK
        now = time.perf_counter() - t0
        for cid, i in list(outstanding.items()):
            if srv.poll(cid)[0] == binding.CASE_DONE:
                done_t[i] = now
                r = srv.result(cid)
                if i in keep:
                    results[i] = r
                del outstanding[cid]
    makespan = time.perf_counter() - t0
    srv.close()
    return dict(done=done_t, makespan=makespan, chunks=chunks, results=results, unstable=unstable)


def serve_sequential(binding, cases, keep=(), every=1):
    """The same cases one at a time in FIFO order through the single-lattice
    handle (its own kernels and CUDA graphs): every `every`-th case, and the
    cases of `keep`. Returns per-case service times (None where not run)."""
    service, results = [None] * len(cases), {}
    for i, w in enumerate(cases):
        if i % every and i not in keep:
            continue
        t0 = time.perf_counter()
        sim = binding.Simulation.from_workload(w)
        sim.step(w['steps'])
        rho, u = sim.fields()
        X, U, _ = sim.markers()
        sim.close()
        service[i] = time.perf_counter() - t0
        if i in keep:
            results[i] = dict(rho=rho, u=u, X=X, U=U)
    return service, results


def fifo_latency(arrivals, service):
    """Completion minus arrival of a one-at-a-time FIFO server."""
    t, lat = 0.0, []
    for a, s in sorted(zip(arrivals, service)):
        t = max(t, a) + s
        lat.append(t - a)
    return lat


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q))


def run_serve(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device('cuda', local)
    dist = init_dist(ws, 'nccl')
    from paper_1704_04551_gb300 import binding, build
    build.build()
    cases = serving_cases(args)
    n = len(cases)
    updates = sum(w['N'] * w['steps'] for w in cases)
    alg_bytes = sum(w['B_step'] * w['steps'] for w in cases)
    keep = tuple(range(0, n, max(1, n // 4)))

    # warm-up: the smallest cases through a server, a few chunks each
    small = sorted(cases, key=lambda w: w['N'])[:3]
    warm = [dict(w, steps=args.serve_chunk * 2) for w in small]
    for _ in range(args.warmup):
        serve_batched(binding, warm, [0.0] * len(warm), args)

    # burst: every case arrives at t = 0
    clocks = ClockSampler(local)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clocks.start()
    time.sleep(0.3)
    burst = serve_batched(binding, cases, [0.0] * n, args, keep)
    clk = clocks.stop()
    burst_s = reduce_max(dist, burst['makespan'], device)
    capacity = n / burst['makespan']

    # Poisson arrivals at 0.9 x the measured batched capacity
    rng = np.random.default_rng(1708)
    arr = np.cumsum(rng.exponential(1.0 / (0.9 * capacity), n))
    arr -= arr[0]
    pois = serve_batched(binding, cases, list(arr), args)

    # sequential per-case solves (same GPU, one case at a time, FIFO); with
    # --serve-seq-every K only every K-th case runs, and the others' service
    # times are estimated at the sample's rate (seconds per lattice update)
    service, seq_res = serve_sequential(binding, cases, keep, args.serve_seq_every)
    ran = [i for i in range(n) if service[i] is not None]
    sec_per_update = sum(service[i] for i in ran) / sum(cases[i]['N'] * cases[i]['steps'] for i in ran)
    service = [s if s is not None else w['N'] * w['steps'] * sec_per_update for s, w in zip(service, cases)]
    seq_s = sum(service)

    # equal accuracy: batched and sequential results of sampled cases
    du = max(float(np.linalg.norm(burst['results'][i]['u'] - seq_res[i]['u']) /
                   max(np.linalg.norm(seq_res[i]['u']), 1e-300)) for i in keep)
    dX = max(float(np.abs(burst['results'][i]['X'] - seq_res[i]['X']).max()) for i in keep)

    lat_burst = [t for t in burst['done']]
    lat_pois = [t - a for t, a in zip(pois['done'], arr)]
    seq_burst = fifo_latency([0.0] * n, service)
    seq_pois = fifo_latency(list(arr), service)
    value = aggregate(updates, burst_s, ws) / 1e6
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / burst['makespan'] / 1e9

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        w0 = cases[0]
        k = 40
        r = time_oracle(w0, k)
        hc = host_cpu()
        cpu = dict(value=r['mlups'], unit=UNIT, cores=r['threads'], kind='oracle',
                   sample=f'{k} coupled steps of serving case 0 ({w0["name"]}) on {r["threads"]} host threads '
                          f'(FP64 C oracle)',
                   seconds=r['seconds'], nproc=hc['nproc'], cpu_model=hc['model'])
    if rank == 0:
        h2d = sum(w['X'].nbytes for w in cases)
        d2h = sum(w['N'] * 4 * 8 + w['X'].nbytes * 2 for w in cases)
        Ls = [w['lattice']['nx'] for w in cases]
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=burst['chunks'], warmup=args.warmup,
            ms_per_step=1e3 * burst['makespan'] / burst['chunks'], higher_is_better=True, scaling='weak',
            vs_baseline=None, dtype='f32', data='synthetic',
            config=dict(workload=f'serving_stream_{n}cases_{args.period_scale:g}x2T',
                        cases=n, seed=1708, lattice_L=[min(Ls), max(Ls)], total_lattice_updates=updates,
                        case_steps=[min(w['steps'] for w in cases), max(w['steps'] for w in cases)],
                        slots=args.serve_slots, chunk_steps=args.serve_chunk,
                        step='one server advance = chunk_steps coupled steps of every admitted case',
                        l2='working set of the admitted cases larger than L2' if sum(w['N'] for w in cases) * 124 > 129e6 else 'working set fits L2',
                        parallelism=f'replicas x{ws}' if ws > 1 else 'single GPU'),
            serving=dict(
                burst=dict(p50_s=pct(lat_burst, 50), p99_s=pct(lat_burst, 99), makespan_s=burst['makespan'],
                           mlups=updates / burst['makespan'] / 1e6, chunks=burst['chunks']),
                poisson=dict(rate_per_s=0.9 * capacity, p50_s=pct(lat_pois, 50), p99_s=pct(lat_pois, 99),
                             makespan_s=pois['makespan'], mlups=updates / pois['makespan'] / 1e6),
                sequential=dict(mlups=updates / seq_s / 1e6, makespan_s=seq_s,
                                burst_p50_s=pct(seq_burst, 50), burst_p99_s=pct(seq_burst, 99),
                                poisson_p50_s=pct(seq_pois, 50), poisson_p99_s=pct(seq_pois, 99),
                                cases_run=len(ran),
                                note='single-lattice handle per case, FIFO; Poisson latencies from the measured service times'
                                     + ('' if len(ran) == n else
                                        f' of {len(ran)} sampled cases (every {args.serve_seq_every}th), the '
                                        'others estimated at the sample\'s seconds per lattice update')),
                speedup_vs_sequential=seq_s / burst['makespan'],
                equal_accuracy=dict(max_rel_l2_u=du, max_abs_dX=dX, cases_compared=len(keep)),
                unstable_cases=burst['unstable'] + pois['unstable']),
            roofline=dict(bound='hbm', achieved=achieved, peak=peak, unit='GB/s', frac=achieved / peak, traffic=None,
                          kernel='whole batched step (all stages, host admission gaps included)',
                          peak_source=f'{peak_kind} hbm_gbs (burst copy)', alg_bytes=alg_bytes),
            cpu_baseline=cpu,
            e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=h2d / burst['chunks'],
                     d2h_bytes_per_step=d2h / burst['chunks'],
                     note='serving is end to end by construction: submission copies from host, results are read back to host inside the timed loop'),
            clocks=dict(sm_mhz=clk['sm_mhz'], sm_max_mhz=clk['sm_max_mhz'], reasons=clk['reasons'],
                        samples=clk['samples']),
            gpu_launches=burst['chunks'] * args.serve_chunk * 7 + 4 * n)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0



def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=1000)
    ap.add_argument('--warmup', type=int, default=20)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--workload', default='tube256',
                    choices=['tube256', 'tube256_f16', 'tube256_bf16', 'tube160', 'tube64', 'shear32', 'mix512',
                             'mix512_f32', 'mix128', 'serve'])
    ap.add_argument('--serve-cases', type=int, default=64)
    ap.add_argument('--period-scale', type=float, default=0.05)
    ap.add_argument('--serve-slots', type=int, default=64)
    ap.add_argument('--serve-chunk', type=int, default=100)
    ap.add_argument('--serve-budget-gb', type=float, default=64.0)
    ap.add_argument('--serve-seq-every', type=int, default=1,
                    help='sequential arm: run every K-th case, estimate the others at the sample\'s rate')
    ap.add_argument('--storage', default=None, choices=[None, 'f32', 'f16', 'bf16'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--ref-max-steps', type=int, default=2)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit('--warmup must be >= 3')
    if args.impl == 'reference':
        return run_reference(args)
    if args.workload == 'serve':
        return run_serve(args)
    return run_ours(args)


if __name__ == '__main__':
    sys.exit(main())
