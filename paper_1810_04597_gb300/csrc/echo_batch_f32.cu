// echo_batch_f32.cu -- batched-run kernels for float storage.
#include "echo_batch_kernels.cuh"

namespace echo {

// The persistent stage kernel calls its phase bodies out of line, so its
// registers are those of the largest body plus the call overhead; with FP32
// storage a bound of 8 blocks per SM (64 registers, a few spills in the EMF
// body) beat 4 and 6 on the 16-torus sweep (27.4 vs 39.6 and 30.9 ms per
// step).  The FP64 bodies need more registers and keep the bound of 4.
template <>
const void *batch_stage_kernel<float>(int mk, bool mlp)
{
    if (mk == 1)
        return mlp ? (const void *)k_batch_stage<1, float, 3, 8> : (const void *)k_batch_stage<1, float, 0, 8>;
    return mlp ? (const void *)k_batch_stage<0, float, 3, 8> : (const void *)k_batch_stage<0, float, 0, 8>;
}

template <int MK>
static void guess_pass(const RunDesc<float> *descs, const BatchPlan *planp, const BatchPlan &P, float gr_f, cudaStream_t s)
{
    // the grid is sized for the whole GPU: the lists' lengths are on the device
    static int resident = 0;
    if (resident == 0)
        resident = tc_resident_ctas((const void *)k_bphase_guess_tc<MK, float>, TC_SMEM);
    k_bphase_guess_tc<MK, float><<<(unsigned)resident, 128, TC_SMEM, s>>>(descs, planp, gr_f);
    k_bphase_clear_lists<float><<<1, 32, 0, s>>>(descs, P.nruns);
}

template <>
void batch_enqueue_guess<float>(int mk, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan, float gr_f,
                            cudaStream_t s)
{
    const RunDesc<float> *d = static_cast<const RunDesc<float> *>(descs);
    if (mk == 1)
        guess_pass<1>(d, plan_dev, plan, gr_f, s);
    else
        guess_pass<0>(d, plan_dev, plan, gr_f, s);
}

template <int MK>
static void phased(bool mlp, const RunDesc<float> *descs, const BatchPlan *planp, const BatchPlan &P, int nruns,
                   const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    k_bphase_scalars<float><<<1, 32, 0, s>>>(descs, nruns, 0, dt, cfl);
    for (int st = 0; st < 3; ++st) {
        for (int p = PH_FILLF0; p <= PH_FILLF2; ++p)
            k_bphase_fill<float><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        if (mlp) {
            guess_pass<MK>(descs, planp, P, ph.gr_f, s);
            k_bphase_c2p<MK, float, 3><<<(unsigned)P.ntiles[PH_C2P], 128, 0, s>>>(descs, planp, ph, guess, st == 0 ? 1 : 0);
        } else {
            k_bphase_c2p<MK, float, 0><<<(unsigned)P.ntiles[PH_C2P], 128, 0, s>>>(descs, planp, ph, guess, st == 0 ? 1 : 0);
        }
        if (st == 0)
            k_bphase_scalars<float><<<1, 32, 0, s>>>(descs, nruns, 1, dt, cfl);
        for (int p = PH_FILLP0; p <= PH_FILLP2; ++p)
            k_bphase_fill<float><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        k_bphase_faces<MK, float><<<(unsigned)P.ntiles[PH_FACES], 128, 0, s>>>(descs, planp, ph);
        k_bphase_emf<MK, float><<<(unsigned)P.ntiles[PH_EMF], 128, 0, s>>>(descs, planp);
        k_bphase_update<MK, float><<<(unsigned)P.ntiles[PH_UPDATE], 128, 0, s>>>(descs, planp, ph, st);
    }
}

template <>
void batch_enqueue_phased<float>(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                              int nruns, const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    const RunDesc<float> *d = static_cast<const RunDesc<float> *>(descs);
    if (mk == 1)
        phased<1>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
    else
        phased<0>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
}

}  // namespace echo
