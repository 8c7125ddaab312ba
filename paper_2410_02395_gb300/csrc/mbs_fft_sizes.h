// Subdomain edge lengths that have compiled FFT pass kernels: every n <= 512
// whose prime factors are 2, 3, 5 and 7 (106 lengths). They are spread over 15
// translation units (mbs_fft_g<k>.cu) of about equal compile cost so that the
// build runs them in parallel. MBS_FFT_GROUP_<k>(X) expands X(n) for every
// length n of group k; MBS_FFT_GROUP_IDS(G) expands G(k) for every group.
#pragma once

#define MBS_FFT_NGROUPS 15
#define MBS_FFT_GROUP_IDS(G) G(0) G(1) G(2) G(3) G(4) G(5) G(6) G(7) G(8) G(9) G(10) G(11) G(12) G(13) G(14)

#define MBS_FFT_GROUP_0(X) X(1) X(20) X(50) X(100) X(168) X(252) X(378) X(512)
#define MBS_FFT_GROUP_1(X) X(18) X(49) X(98) X(162) X(250) X(375) X(504)
#define MBS_FFT_GROUP_2(X) X(16) X(48) X(96) X(160) X(245) X(360) X(500)
#define MBS_FFT_GROUP_3(X) X(15) X(45) X(90) X(150) X(243) X(350) X(490)
#define MBS_FFT_GROUP_4(X) X(14) X(42) X(84) X(147) X(240) X(343) X(486)
#define MBS_FFT_GROUP_5(X) X(12) X(40) X(81) X(144) X(225) X(336) X(480)
#define MBS_FFT_GROUP_6(X) X(10) X(36) X(80) X(140) X(224) X(324) X(450)
#define MBS_FFT_GROUP_7(X) X(9) X(35) X(75) X(135) X(216) X(320) X(448)
#define MBS_FFT_GROUP_8(X) X(8) X(32) X(72) X(128) X(210) X(315) X(441)
#define MBS_FFT_GROUP_9(X) X(7) X(30) X(70) X(126) X(200) X(300) X(432)
#define MBS_FFT_GROUP_10(X) X(6) X(28) X(64) X(125) X(196) X(294) X(420)
#define MBS_FFT_GROUP_11(X) X(5) X(27) X(63) X(120) X(192) X(288) X(405)
#define MBS_FFT_GROUP_12(X) X(4) X(25) X(60) X(112) X(189) X(280) X(400)
#define MBS_FFT_GROUP_13(X) X(3) X(24) X(56) X(108) X(180) X(270) X(392)
#define MBS_FFT_GROUP_14(X) X(2) X(21) X(54) X(105) X(175) X(256) X(384)
