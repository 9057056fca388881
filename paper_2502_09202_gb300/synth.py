"""Seeded synthetic luma video: the inputs shared by the CUDA path and the oracle.

This module only makes test video and its planted ground truth. It holds none of
the analyser's arithmetic (no pyramid, search, correlation or decision rule).

Every frame is a pure function of (clip spec, frame index): ``Clip.frame(t)`` can
be called in any order, so a clip of any length is streamed without holding it.

Conventions (shared by every config):

* Scenes: a world canvas (background) seen through a camera that pans by an
  integer number of pixels per time unit, plus rectangular textured objects that
  move by an integer number of pixels per time unit and wrap around the frame.
  Textures are uniform noise drawn per ``cell`` x ``cell`` square.
* Time units: a progressive clip moves once per frame; an interlaced clip once per
  field (even rows of frame t at field time 2t for top-field-first, odd rows at
  2t+1; swapped for bottom-field-first); a 3:2 pulldown clip once per film frame.
* 3:2 pulldown: video frame k has cadence position c = (k - phase) mod 5 and
  unit u = (k - phase) div 5; its (top, bottom) fields show film frames
  A A / B B / B C / C D / D D of unit u for c = 0..4 (A = 4u, ..., D = 4u+3).
* A linear dissolve of L frames starting at s blends frame s+i as
  (a*(L-1-i) + b*i + (L-1)//2) // (L-1): frame s is the outgoing shot, frame
  s+L-1 the incoming one, so the transition spans K = L-1 frame steps.
* Flash: +80 luma on one frame, clipped to 255.
* Noise: a zero-mean Gaussian of standard deviation sigma, quantised to integers
  through a 65536-entry inverse-CDF table indexed by 16-bit PCG64 draws, added per
  pixel after everything else and clipped to 0..255.
"""
from __future__ import annotations

import math
import statistics
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

PROGRESSIVE, TFF, BFF, PULLDOWN = "progressive", "tff", "bff", "pulldown"
STRUCTURES = (PROGRESSIVE, TFF, BFF, PULLDOWN)
FLASH_DELTA = 80


def _rng(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(k) & 0xFFFFFFFF for k in keys]))


@lru_cache(maxsize=16)
def _noise_table(sigma: float) -> np.ndarray:
    nd = statistics.NormalDist(0.0, sigma)
    q = np.array([nd.inv_cdf((i + 0.5) / 65536.0) for i in range(65536)])
    return np.rint(q).astype(np.int16)


def _cell_noise(rng: np.random.Generator, h: int, w: int, lo: int, hi: int, cell: int) -> np.ndarray:
    ch, cw = -(-h // cell), -(-w // cell)
    c = rng.integers(lo, hi + 1, size=(ch, cw), dtype=np.int16)
    return np.repeat(np.repeat(c, cell, axis=0), cell, axis=1)[:h, :w]


@dataclass
class SceneStyle:
    """How a clip's scenes look and move (per time unit of the clip's structure)."""

    n_objects: tuple[int, int] = (6, 6)
    obj_size: tuple[float, float] = (0.10, 0.25)   # fraction of the frame side
    obj_speed: int = 4                             # |v| per axis, px per time unit
    obj_range: tuple[int, int] = (0, 255)          # object texture values
    cell: int = 4                                  # texture cell size in px
    pan_x: tuple[int, int] = (1, 1)                # camera pan range per axis
    pan_y: tuple[int, int] = (0, 0)
    bg_kind: str = "gradient"                      # "gradient" | "textured" | "lowcontrast"
    bg_lo: int = 30
    bg_hi: int = 220


@dataclass
class Scene:
    world: np.ndarray           # int16 background canvas, wraps in both axes
    pan: tuple[int, int]        # (px, py) per time unit
    origin: tuple[int, int]
    objects: list               # (texture int16 h x w, x0, y0, vx, vy)


def make_scene(seed: int, key: int, width: int, height: int, style: SceneStyle) -> Scene:
    rng = _rng(seed, 7919, key)
    ww, wh = width + 512, height + 256
    if style.bg_kind == "gradient":
        xs = np.arange(ww, dtype=np.float64)
        g = np.rint(style.bg_lo + (style.bg_hi - style.bg_lo) * xs / (ww - 1)).astype(np.int16)
        world = np.broadcast_to(g, (wh, ww)).copy()
    elif style.bg_kind == "textured":
        xs = np.arange(ww, dtype=np.float64)
        g = np.rint(60 + 120 * xs / (ww - 1)).astype(np.int16)
        world = g[None, :] + _cell_noise(rng, wh, ww, -40, 40, max(style.cell, 4))
    elif style.bg_kind == "lowcontrast":
        world = _cell_noise(rng, wh, ww, style.bg_lo, style.bg_hi, style.cell)
    else:
        raise ValueError(style.bg_kind)
    px = int(rng.integers(style.pan_x[0], style.pan_x[1] + 1)) * (1 if rng.integers(2) else -1)
    py = int(rng.integers(style.pan_y[0], style.pan_y[1] + 1)) * (1 if rng.integers(2) else -1)
    origin = (int(rng.integers(0, ww)), int(rng.integers(0, wh)))
    objs = []
    n = int(rng.integers(style.n_objects[0], style.n_objects[1] + 1))
    side = min(width, height)
    for _ in range(n):
        ow = max(8, int(side * rng.uniform(*style.obj_size)))
        oh = max(8, int(side * rng.uniform(*style.obj_size)))
        tex = _cell_noise(rng, oh, ow, style.obj_range[0], style.obj_range[1], style.cell)
        x0 = int(rng.integers(0, width))
        y0 = int(rng.integers(0, height))
        vx = int(rng.integers(-style.obj_speed, style.obj_speed + 1))
        vy = int(rng.integers(-style.obj_speed, style.obj_speed + 1))
        objs.append((tex, x0, y0, vx, vy))
    return Scene(world=world, pan=(px, py), origin=origin, objects=objs)


def render(scene: Scene, tau: int, width: int, height: int) -> np.ndarray:
    """The scene at integer time ``tau`` as an int16 height x width image."""
    wh, ww = scene.world.shape
    cx = (scene.origin[0] + scene.pan[0] * tau) % ww
    cy = (scene.origin[1] + scene.pan[1] * tau) % wh
    rows = (cy + np.arange(height)) % wh
    cols = (cx + np.arange(width)) % ww
    if cy + height <= wh:
        img = scene.world[cy:cy + height]
    else:
        img = scene.world.take(rows, axis=0)
    if cx + width <= ww:
        img = img[:, cx:cx + width].copy()
    else:
        img = img.take(cols, axis=1)
    for tex, x0, y0, vx, vy in scene.objects:
        oh, ow = tex.shape
        # objects wrap over a period of (frame side + object side) so they re-enter
        x = (x0 + vx * tau) % (width + ow) - ow
        y = (y0 + vy * tau) % (height + oh) - oh
        xa, xb = max(x, 0), min(x + ow, width)
        ya, yb = max(y, 0), min(y + oh, height)
        if xa < xb and ya < yb:
            img[ya:yb, xa:xb] = tex[ya - y:yb - y, xa - x:xb - x]
    return img


@dataclass
class ClipSpec:
    width: int
    height: int
    nframes: int
    fps: float
    structure: str
    seed: int
    sigma: float
    style: SceneStyle
    cuts: list = field(default_factory=list)        # first frame of each new shot
    dissolves: list = field(default_factory=list)   # (start s, length L)
    flashes: list = field(default_factory=list)     # frame indices
    pulldown_phase: int = 0
    flicker: float = 0.0                            # amplitude (luma) of a sinusoidal flicker
    flicker_hz: float = 0.0
    name: str = ""

    @property
    def pixels(self) -> int:
        return self.width * self.height


class Clip:
    """Random-access frame source for one ClipSpec, with its ground truth."""

    def __init__(self, spec: ClipSpec):
        self.spec = spec
        s = spec
        # shot timeline: (first frame of the shot's scene, scene key)
        starts = sorted([(c, "cut") for c in s.cuts] + [(d[0], "dis", d[1]) for d in s.dissolves])
        self._segments = [(0, 0)]      # (frame where the scene becomes the program, scene key)
        self._blends = []              # (s, L, key_from, key_to)
        key = 0
        for ev in starts:
            if ev[1] == "cut":
                key += 1
                self._segments.append((ev[0], key))
            else:
                st, L = ev[0], ev[2]
                self._blends.append((st, L, key, key + 1))
                key += 1
                self._segments.append((st + L - 1, key))
        self._scene_cache: dict[int, Scene] = {}
        self._noise = _noise_table(float(s.sigma)) if s.sigma > 0 else None

    # ---- ground truth -------------------------------------------------------
    def truth(self) -> dict:
        s = self.spec
        fo = {TFF: "tff", BFF: "bff"}.get(s.structure, "none")
        return {
            "cuts": sorted(s.cuts),
            "dissolves": sorted((st, L - 1) for st, L in s.dissolves),
            "flashes": sorted(s.flashes),
            "structure": s.structure,
            "field_order": fo,
            "pulldown_phase": s.pulldown_phase if s.structure == PULLDOWN else -1,
            "shot_starts": [seg[0] for seg in self._segments],
        }

    # ---- rendering ----------------------------------------------------------
    def _scene(self, key: int) -> Scene:
        sc = self._scene_cache.get(key)
        if sc is None:
            if len(self._scene_cache) > 4:
                self._scene_cache.pop(next(iter(self._scene_cache)))
            sc = make_scene(self.spec.seed, key, self.spec.width, self.spec.height, self.spec.style)
            self._scene_cache[key] = sc
        return sc

    def _program(self, t: int, tau: int, flick_time: float | None) -> np.ndarray:
        s = self.spec
        for st, L, ka, kb in self._blends:
            if st < t < st + L - 1:
                i = t - st
                a = render(self._scene(ka), tau, s.width, s.height).astype(np.int32)
                b = render(self._scene(kb), tau, s.width, s.height).astype(np.int32)
                img = (a * (L - 1 - i) + b * i + (L - 1) // 2) // (L - 1)
                break
        else:
            key = 0
            for start, k in self._segments:
                if start <= t:
                    key = k
            img = render(self._scene(key), tau, s.width, s.height).astype(np.int32)
        if s.flicker and flick_time is not None:
            img = img + int(round(s.flicker * math.sin(2.0 * math.pi * s.flicker_hz * flick_time)))
        return img

    def frame(self, t: int) -> np.ndarray:
        """Frame t as a C-contiguous uint8 (height, width) array."""
        s = self.spec
        if s.structure == PROGRESSIVE:
            img = self._program(t, t, t / s.fps)
        elif s.structure in (TFF, BFF):
            first, second = self._program(t, 2 * t, t / s.fps), self._program(t, 2 * t + 1, t / s.fps)
            img = np.empty_like(first)
            top, bot = (first, second) if s.structure == TFF else (second, first)
            img[0::2] = top[0::2]
            img[1::2] = bot[1::2]
        elif s.structure == PULLDOWN:
            c = (t - s.pulldown_phase) % 5
            u = (t - s.pulldown_phase) // 5
            top_f, bot_f = {0: (0, 0), 1: (1, 1), 2: (1, 2), 3: (2, 3), 4: (3, 3)}[c]
            nt, nb = 4 * u + top_f, 4 * u + bot_f
            film_fps = s.fps * 4.0 / 5.0
            top = self._program(t, nt, nt / film_fps)
            img = top
            if nb != nt:
                bot = self._program(t, nb, nb / film_fps)
                img = top.copy()
                img[1::2] = bot[1::2]
        else:
            raise ValueError(s.structure)
        if t in s.flashes:
            img = img + FLASH_DELTA
        if self._noise is not None:
            r = _rng(s.seed, 104729, t).integers(0, 65536, size=img.shape, dtype=np.uint16)
            img = img + self._noise[r]
        return np.clip(img, 0, 255).astype(np.uint8)

    def frames(self, start: int = 0, stop: int | None = None) -> np.ndarray:
        stop = self.spec.nframes if stop is None else stop
        out = np.empty((stop - start, self.spec.height, self.spec.width), np.uint8)
        for i, t in enumerate(range(start, stop)):
            out[i] = self.frame(t)
        return out


# ---- event placement ----------------------------------------------------------

def _place_events(rng, nframes, gap_range, n_dissolves, dis_len, flash_every, guard, structure, phase):
    """Shot boundaries every gap_range frames; some become dissolves; flashes away from them."""
    bounds = []
    t = int(rng.integers(gap_range[0], gap_range[1] + 1))
    while t < nframes - gap_range[0] // 2:
        if structure == PULLDOWN:
            while (t - phase) % 5 not in (0, 1):
                t += 1
        bounds.append(t)
        t += int(rng.integers(gap_range[0], gap_range[1] + 1))
    bounds = [b for b in bounds if b < nframes - 2 * guard]
    dis_idx = set()
    if n_dissolves and bounds:
        dis_idx = set(int(i) for i in rng.choice(len(bounds), size=min(n_dissolves, len(bounds)), replace=False))
    cuts, dissolves = [], []
    for i, b in enumerate(bounds):
        if i in dis_idx:
            dissolves.append((b - (dis_len - 1), dis_len))
        else:
            cuts.append(b)
    flashes = []
    if flash_every and nframes > 2 * guard + 1:
        busy = []
        for c in cuts:
            busy.append((c - 1, c))
        for st, L in dissolves:
            busy.append((st, st + L - 1))
        for k in range(max(1, nframes // flash_every)):
            for _ in range(200):
                f = int(rng.integers(guard, nframes - guard))
                if all(f < a - guard or f > b + guard for a, b in busy) and all(abs(f - g) > guard for g in flashes):
                    flashes.append(f)
                    busy.append((f, f))
                    break
    return sorted(cuts), sorted(dissolves), sorted(flashes)


# ---- the five workloads ----------------------------------------------------------

KMAX_GUARD = 8 + 3


def config_small(seed: int = 0) -> ClipSpec:
    """320x180, 64 frames, progressive, 25 fps: cuts at 20 and 41, a 5-frame dissolve from 50."""
    style = SceneStyle(n_objects=(6, 6), obj_size=(0.15, 0.35), obj_speed=4, cell=8,
                       pan_x=(1, 1), pan_y=(0, 0), bg_kind="gradient")
    return ClipSpec(320, 180, 64, 25.0, PROGRESSIVE, seed, 2.0, style,
                    cuts=[20, 41], dissolves=[(50, 5)], flashes=[], name="small-320x180-prog")


def config_interlaced(seed: int = 1, nframes: int = 1500, width: int = 1920, height: int = 1080) -> ClipSpec:
    """1920x1080, 1500 frames, 25 fps, top field first, objects up to 16 px/field,
    cuts every 150-250 frames, three 8-frame dissolves, one flash per 300 frames."""
    rng = _rng(seed, 31)
    style = SceneStyle(n_objects=(8, 12), obj_size=(0.10, 0.30), obj_speed=16, cell=8,
                       pan_x=(0, 0), pan_y=(0, 0), bg_kind="textured")
    cuts, dis, fl = _place_events(rng, nframes, (150, 250), 3, 8, 300, KMAX_GUARD, TFF, 0)
    return ClipSpec(width, height, nframes, 25.0, TFF, seed, 4.0, style, cuts=cuts, dissolves=dis,
                    flashes=fl, name=f"interlaced-tff-{width}x{height}")


def config_pulldown(seed: int = 2, nframes: int = 1800, width: int = 1920, height: int = 1080) -> ClipSpec:
    """1920x1080, 1800 frames, 29.97 fps, 3:2 pulldown of a 24p source with a seeded
    phase; low contrast (96..160), +-6 flicker at 0.7 Hz, pan up to 24 px per film
    frame, sigma 6, 4 cuts."""
    rng = _rng(seed, 37)
    phase = int(rng.integers(0, 5))
    style = SceneStyle(n_objects=(3, 5), obj_size=(0.10, 0.25), obj_speed=6, obj_range=(96, 160),
                       cell=8, pan_x=(8, 24), pan_y=(0, 6), bg_kind="lowcontrast", bg_lo=96, bg_hi=160)
    gap = (nframes // 5 - 40, nframes // 5 + 40)
    cuts, dis, fl = _place_events(rng, nframes, gap, 0, 0, 0, KMAX_GUARD, PULLDOWN, phase)
    cuts = cuts[:4]
    return ClipSpec(width, height, nframes, 30000.0 / 1001.0, PULLDOWN, seed, 6.0, style, cuts=cuts,
                    dissolves=dis, flashes=fl, pulldown_phase=phase, flicker=6.0, flicker_hz=0.7,
                    name=f"pulldown-{width}x{height}")


RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080), (2048, 1080), (3840, 2160))


def _mixed_clip(rng, seed: int, length_range: tuple[int, int], resolutions=RESOLUTIONS) -> ClipSpec:
    w, h = resolutions[int(rng.integers(0, len(resolutions)))]
    n = int(rng.integers(length_range[0], length_range[1] + 1))
    structure = STRUCTURES[int(rng.integers(0, 4))]
    phase = int(rng.integers(0, 5))
    scale = w / 1920.0
    if structure == PULLDOWN:
        style = SceneStyle(n_objects=(3, 5), obj_size=(0.10, 0.25), obj_speed=max(1, int(6 * scale)),
                           obj_range=(96, 160), cell=8, pan_x=(max(1, int(8 * scale)), max(1, int(24 * scale))),
                           pan_y=(0, 4), bg_kind="lowcontrast", bg_lo=96, bg_hi=160)
        fps = 30000.0 / 1001.0
    else:
        style = SceneStyle(n_objects=(6, 10), obj_size=(0.10, 0.30), obj_speed=max(2, int(16 * scale)),
                           cell=8, pan_x=(0, 0), pan_y=(0, 0), bg_kind="textured")
        fps = 25.0
    cuts, dis, fl = _place_events(rng, n, (40, 120), 1, 5, 150, KMAX_GUARD, structure, phase)
    return ClipSpec(w, h, n, fps, structure, seed, 4.0, style, cuts=cuts, dissolves=dis, flashes=fl,
                    pulldown_phase=phase, name=f"mixed-{structure}-{w}x{h}-{n}")


def config_batched(seed: int = 3, nclips: int = 64, length_range=(60, 600), resolutions=RESOLUTIONS) -> list[ClipSpec]:
    """64 clips, resolutions uniform over RESOLUTIONS, lengths 60..600, structure uniform."""
    rng = _rng(seed, 41)
    return [_mixed_clip(rng, seed * 1000 + i, length_range, resolutions) for i in range(nclips)]


def config_served(seed: int = 4, nrequests: int = 512, rate_hz: float = 40.0, length_range=(30, 300),
                  resolutions=RESOLUTIONS) -> list[tuple[float, ClipSpec]]:
    """512 requests with Poisson arrivals at 40/s; clips drawn as in the batched workload."""
    rng = _rng(seed, 43)
    t = 0.0
    out = []
    for i in range(nrequests):
        t += float(rng.exponential(1.0 / rate_hz))
        out.append((t, _mixed_clip(rng, seed * 100000 + i, length_range, resolutions)))
    return out


def random_frame(seed: int, width: int, height: int, cell: int = 1) -> np.ndarray:
    """i.i.d. (or cell-constant) uniform noise frame; used by shape and edge-case tests."""
    rng = _rng(seed, 53)
    return _cell_noise(rng, height, width, 0, 255, cell).astype(np.uint8)


def shifted_pair(seed: int, width: int, height: int, sx: int, sy: int, cell: int = 1):
    """Two crops of one noise texture, the second displaced so that I(p) = J(p + (sx, sy))."""
    rng = _rng(seed, 59)
    pad = max(abs(sx), abs(sy)) + 1
    big = _cell_noise(rng, height + 2 * pad, width + 2 * pad, 0, 255, cell).astype(np.uint8)
    i_img = big[pad:pad + height, pad:pad + width].copy()
    j_img = big[pad - sy:pad - sy + height, pad - sx:pad - sx + width].copy()
    return i_img, j_img
